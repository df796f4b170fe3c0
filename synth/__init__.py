"""Seeded synthetic inputs: DNA texts, IUPAC class patterns and planted copies.

This module is the one thing the oracle side (tests, CPU baseline) and the CUDA
side share.  It holds none of the matching method's arithmetic: no symbol
codes, no dictionary, no sums.  It writes ASCII texts and pattern strings; the
only biology it knows is which letters each IUPAC class letter stands for,
which it needs to plant copies with an exact number of mismatches.

The workloads stand in for the paper's human chromosome 2 (GRCh37, 243 Mbp;
Sec. 3), which is not available here:

* ``uniform_text``   i.i.d. uniform ACGT (numpy ``default_rng(seed)``);
* ``markov_text``    an order-2 Markov chain with CpG depletion, calibrated to
                     a 41 % GC stationary content, generated by ``markov.c`` in
                     1 Mbp blocks each keyed by (seed, block) so that it is
                     reproducible at any thread count;
* ``random_pattern`` m positions, a given number of them drawn (without
                     replacement) as two- or three-letter IUPAC classes
                     (M R W S Y K V H D B), the rest uniform single letters;
* ``plant``          non-overlapping copies of a pattern, each a concrete
                     instance of it with exactly s positions replaced by a
                     letter outside that position's class.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "markov.c")
_LIB = os.path.join(_HERE, "libsynth.so")
_lock = threading.Lock()
_lib = None

LETTERS = "ACGT"
# IUPAC class letters and the DNA letters each stands for.
IUPAC = {
    "A": "A", "C": "C", "G": "G", "T": "T",
    "M": "AC", "R": "AG", "W": "AT", "S": "CG", "Y": "CT", "K": "GT",
    "V": "ACG", "H": "ACT", "D": "AGT", "B": "CGT", "N": "ACGT",
}
TWO_THREE_LETTER = "MRWSYKVHDB"


def build(force: bool = False) -> str:
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread",
                           "-Wall", "-o", tmp, _SRC])
    os.replace(tmp, _LIB)
    return _LIB


def _clib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            L.synth_markov.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64,
                                       ctypes.c_void_p, ctypes.c_int]
            L.synth_markov_range.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64,
                                             ctypes.c_uint64, ctypes.c_void_p, ctypes.c_int]
            L.synth_gc_fraction.argtypes = [ctypes.c_void_p, ctypes.c_uint64]
            L.synth_gc_fraction.restype = ctypes.c_double
            _lib = L
    return _lib


# ---------------------------------------------------------------- texts ----

_ASCII = np.frombuffer(LETTERS.encode(), dtype=np.uint8)


def uniform_text(n: int, seed: int) -> np.ndarray:
    """i.i.d. uniform ACGT as a uint8 ASCII array."""
    rng = np.random.default_rng(seed)
    return _ASCII[rng.integers(0, 4, size=n, dtype=np.uint8)]


def markov_table(gc: float = 0.41) -> np.ndarray:
    """16 x 4 transition probabilities P(x_t | x_{t-2}, x_{t-1}).

    Base weights A = T = 0.295, C = G = 0.205; a G after a C is weighted by
    0.25 (CpG depletion); a fixed factor in [0.85, 1.15] per (context, letter)
    makes the chain genuinely order 2; finally C and G are scaled by one
    common factor, found by bisection, so that the stationary GC fraction
    equals ``gc``.
    """
    base = np.array([0.295, 0.205, 0.205, 0.295])
    wiggle = np.random.default_rng(20161118).uniform(0.85, 1.15, size=(16, 4))

    def table(g):
        P = np.empty((16, 4))
        for ctx in range(16):
            x1 = ctx & 3
            w = base * wiggle[ctx]
            w = w * np.array([1.0, g, g, 1.0])
            if x1 == 1:        # previous letter C
                w[2] *= 0.25   # CpG depletion
            P[ctx] = w / w.sum()
        return P

    def stationary_gc(P):
        T = np.zeros((16, 16))
        for ctx in range(16):
            x1 = ctx & 3
            for x in range(4):
                T[ctx, 4 * x1 + x] += P[ctx, x]
        pi = np.full(16, 1 / 16)
        for _ in range(2000):
            pi = pi @ T
        pi /= pi.sum()
        return float(sum(pi[c] for c in range(16) if (c & 3) in (1, 2)))

    lo, hi = 0.5, 3.0
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        if stationary_gc(table(mid)) < gc:
            lo = mid
        else:
            hi = mid
    return table(0.5 * (lo + hi))


def _thresholds(P: np.ndarray) -> np.ndarray:
    cum = np.cumsum(P, axis=1)[:, :3]
    return np.clip(np.round(cum * 2.0 ** 32), 0, 2 ** 32 - 1).astype(np.uint32).reshape(-1)


_THRESH: dict[float, np.ndarray] = {}


def markov_text(n: int, seed: int, gc: float = 0.41, out: np.ndarray | None = None,
                threads: int = 0, start: int = 0) -> np.ndarray:
    """Symbols [start, start + n) of the order-2 Markov ACGT text with this seed
    (uint8 ASCII), written into ``out`` if given (any writable contiguous uint8
    buffer, e.g. pinned host memory).  Any range of the same seed agrees with
    the corresponding slice of the whole text."""
    if out is None:
        out = np.empty(n, dtype=np.uint8)
    assert out.dtype == np.uint8 and out.flags.c_contiguous and out.size >= n
    if gc not in _THRESH:
        _THRESH[gc] = np.ascontiguousarray(_thresholds(markov_table(gc)))
    thr = _THRESH[gc]
    _clib().synth_markov_range(out.ctypes.data, start, n, seed, thr.ctypes.data,
                               threads or (os.cpu_count() or 1))
    return out[:n]


def gc_fraction(text: np.ndarray) -> float:
    t = np.ascontiguousarray(text, dtype=np.uint8)
    return _clib().synth_gc_fraction(t.ctypes.data, t.size)


# ------------------------------------------------------------- patterns ----

def random_pattern(m: int, n_class: int, rng: np.random.Generator) -> str:
    """m symbols; ``n_class`` positions (without replacement) are two- or
    three-letter classes chosen uniformly, the rest uniform single letters."""
    sym = [LETTERS[i] for i in rng.integers(0, 4, size=m)]
    if n_class:
        pos = rng.choice(m, size=min(n_class, m), replace=False)
        for p in pos:
            sym[int(p)] = TWO_THREE_LETTER[int(rng.integers(0, len(TWO_THREE_LETTER)))]
    return "".join(sym)


def instance(pattern: str, subs: int, rng: np.random.Generator) -> str:
    """A concrete text string matching ``pattern`` except at exactly ``subs``
    positions, which get a letter outside that position's class.  Positions
    whose class is N or whose symbol is unknown are never chosen for a
    substitution (N has no letter outside it)."""
    out = []
    for ch in pattern:
        letters = IUPAC.get(ch.upper(), "")
        out.append(letters[int(rng.integers(0, len(letters)))] if letters else "A")
    can = [j for j, ch in enumerate(pattern) if 0 < len(IUPAC.get(ch.upper(), "")) < 4]
    if subs > len(can):
        raise ValueError("more substitutions than substitutable positions")
    for j in rng.choice(len(can), size=subs, replace=False) if subs else []:
        j = can[int(j)]
        outside = [a for a in LETTERS if a not in IUPAC[pattern[j].upper()]]
        out[j] = outside[int(rng.integers(0, len(outside)))]
    return "".join(out)


class Occupancy:
    """Non-overlapping intervals [a, b) already used by planted copies, kept
    sorted by start."""

    def __init__(self):
        self.iv: list[tuple[int, int]] = []

    def free(self, a: int, b: int) -> bool:
        import bisect
        i = bisect.bisect_left(self.iv, (a, b))
        if i > 0 and self.iv[i - 1][1] > a:
            return False
        return i == len(self.iv) or self.iv[i][0] >= b

    def take(self, a: int, b: int):
        import bisect
        bisect.insort(self.iv, (a, b))


def plant(text: np.ndarray, pattern: str, count: int, s_max: int,
          rng: np.random.Generator, occ: Occupancy | None = None,
          s_min: int = 0) -> list[tuple[int, int]]:
    """Write ``count`` non-overlapping noisy copies of ``pattern`` into ``text``
    (uint8 ASCII, in place); copy q gets s_q substitutions, s_q uniform in
    [s_min, s_max].  Returns [(location, s_q)] sorted by location."""
    occ = occ if occ is not None else Occupancy()
    n, m = text.size, len(pattern)
    out = []
    for _ in range(count):
        for _try in range(10000):
            loc = int(rng.integers(0, n - m + 1))
            if occ.free(loc, loc + m):
                break
        else:
            raise RuntimeError("could not place a planted copy")
        s = int(rng.integers(s_min, s_max + 1))
        text[loc:loc + m] = np.frombuffer(instance(pattern, s, rng).encode(), dtype=np.uint8)
        occ.take(loc, loc + m)
        out.append((loc, s))
    return sorted(out)


def log_uniform_lengths(count: int, lo: int, hi: int, rng: np.random.Generator) -> np.ndarray:
    """round(exp(U(ln lo, ln hi))), clipped to [lo, hi]."""
    x = np.exp(rng.uniform(math.log(lo), math.log(hi), size=count))
    return np.clip(np.round(x), lo, hi).astype(np.int64)


def poisson_arrivals(rate: float, duration: float, rng: np.random.Generator) -> np.ndarray:
    """Arrival times (s) of a Poisson process of the given rate over [0, duration)."""
    t, out = 0.0, []
    while True:
        t += float(rng.exponential(1.0 / rate))
        if t >= duration:
            return np.array(out)
        out.append(t)
