"""Oracle for k-mismatch character-class pattern matching.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product package
never imports it and it never imports the product package; the two share no
code.  The only inputs both sides see come from ``synth`` (seeded generators).

Contents
--------
``pm_oracle.c``      the paper's method written out plainly in C: Table 1 and
                     Table 2 codes, the Table 3 dictionary, the index
                     ``(p[j] << 2) OR t[i+j-1]`` of Sec. 2.3, the sum of Eq. 4
                     with the early stop of Sec. 2.4/2.5, and the Sec. 2.6 split
                     into overlapping pieces, one per thread.
``linhart_shamir.py`` the prime-coding method of Sec. 1.3 (Eq. 1-3) in exact
                     Python integers: an independent route to the same counts,
                     used as a pin for tiny inputs.

Every function here is pinned by ``tests/test_oracle.py`` against the worked
examples (Sec. 1.1; Sec. 2.5 and Table 4), Table 2's class column, the
prime-product test, brute force and invariants; none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pm_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, E_ARG, E_SYMBOL, E_OVERFLOW, E_NOMEM = 0, -1, -2, -3, -4


class OracleError(RuntimeError):
    pass


def build(force: bool = False) -> str:
    """Compile ``pm_oracle.c`` into ``liboracle.so`` with gcc (plain C, -O2)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread",
                           "-Wall", "-Wextra", "-o", tmp, _SRC])
    os.replace(tmp, _LIB)
    return _LIB


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            c_p = ctypes.c_char_p
            u64, i64, u32 = ctypes.c_uint64, ctypes.c_int64, ctypes.c_uint32
            vp = ctypes.c_void_p
            L.oracle_text_code.argtypes = [ctypes.c_int]
            L.oracle_pattern_code.argtypes = [ctypes.c_int]
            L.oracle_lindex.argtypes = [ctypes.c_int, ctypes.c_int]
            L.oracle_table3.restype = ctypes.POINTER(ctypes.c_uint8)
            L.oracle_count_unknown.argtypes = [c_p, u32]
            L.oracle_window_trace.argtypes = [vp, u64, c_p, u32, u64, i64, ctypes.c_int, vp, vp]
            L.oracle_counts.argtypes = [vp, u64, c_p, u32, vp, ctypes.POINTER(i64)]
            L.oracle_counts_at.argtypes = [vp, u64, c_p, u32, vp, u64, vp]
            L.oracle_counts_unknown_text.argtypes = [vp, u64, c_p, u32, vp]
            L.oracle_search_unknown_text.argtypes = [vp, u64, c_p, u32, i64, vp, vp, u64,
                                                     ctypes.POINTER(u64)]
            L.oracle_search.argtypes = [vp, u64, c_p, u32, i64, ctypes.c_int, ctypes.c_int,
                                        vp, vp, vp, u64, ctypes.POINTER(u64),
                                        ctypes.POINTER(i64)]
            _lib = L
    return _lib


def _text_buf(text) -> tuple[np.ndarray, int]:
    """Accept bytes, str, or a uint8 numpy array; return a contiguous uint8 array."""
    if isinstance(text, str):
        text = text.encode("ascii")
    if isinstance(text, (bytes, bytearray, memoryview)):
        arr = np.frombuffer(bytes(text), dtype=np.uint8)
    else:
        arr = np.ascontiguousarray(np.asarray(text, dtype=np.uint8))
    return arr, int(arr.size)


def _pat(pattern) -> bytes:
    if isinstance(pattern, str):
        return pattern.encode("ascii")
    return bytes(pattern)


def text_code(ch: str) -> int:
    """Table 1 code of one text symbol, or -1."""
    return lib().oracle_text_code(ord(ch))


def pattern_code(ch: str) -> int:
    """Table 2 code of one pattern symbol (unknown -> 15)."""
    return lib().oracle_pattern_code(ord(ch))


def lindex(pcode: int, tcode: int) -> int:
    """Sec. 2.3 index ``(p << 2) OR t``."""
    return lib().oracle_lindex(pcode, tcode)


def table3() -> np.ndarray:
    """The 64-entry dictionary L of Table 3 as the oracle holds it."""
    p = lib().oracle_table3()
    return np.array([p[i] for i in range(64)], dtype=np.uint8)


def count_unknown(pattern) -> int:
    """Number of pattern symbols that Table 2 does not list (coded 1111)."""
    pb = _pat(pattern)
    return lib().oracle_count_unknown(pb, len(pb))


def window_trace(text, pattern, location: int, k: int, early_exit: bool = True):
    """Step 4 of Sec. 2.5 for one 0-based window: the l indices looked up, in
    order, and the dictionary values read, stopping once the sum exceeds k."""
    arr, n = _text_buf(text)
    pb = _pat(pattern)
    m = len(pb)
    lv = np.zeros(max(m, 1), dtype=np.int32)
    vv = np.zeros(max(m, 1), dtype=np.int32)
    c = lib().oracle_window_trace(arr.ctypes.data, n, pb, m, int(location), int(k),
                                  1 if early_exit else 0, lv.ctypes.data, vv.ctypes.data)
    if c < 0:
        raise OracleError(f"oracle_window_trace failed: {c}")
    return lv[:c].tolist(), vv[:c].tolist()


def counts(text, pattern) -> np.ndarray:
    """Full Eq. 4 sums, no early stop, for every window 0..n-m (small inputs)."""
    arr, n = _text_buf(text)
    pb = _pat(pattern)
    m = len(pb)
    nwin = max(n - m + 1, 0)
    out = np.zeros(max(nwin, 1), dtype=np.uint32)
    bad = ctypes.c_int64(-1)
    rc = lib().oracle_counts(arr.ctypes.data, n, pb, m, out.ctypes.data, ctypes.byref(bad))
    if rc == E_SYMBOL:
        raise OracleError(f"text symbol outside Table 1 at offset {bad.value}")
    if rc != OK:
        raise OracleError(f"oracle_counts failed: {rc}")
    return out[:nwin]


def counts_at(text, pattern, locations) -> np.ndarray:
    """Full Eq. 4 sums at the given 0-based window locations."""
    arr, n = _text_buf(text)
    pb = _pat(pattern)
    locs = np.ascontiguousarray(np.asarray(locations, dtype=np.uint64))
    out = np.zeros(max(locs.size, 1), dtype=np.uint32)
    rc = lib().oracle_counts_at(arr.ctypes.data, n, pb, len(pb), locs.ctypes.data,
                                locs.size, out.ctypes.data)
    if rc != OK:
        raise OracleError(f"oracle_counts_at failed: {rc}")
    return out[:locs.size]


def search(text, pattern, k: int, early_exit: bool = True, threads: int = 0,
           split_at=None) -> tuple[np.ndarray, np.ndarray]:
    """All 0-based locations whose Eq. 4 sum is <= k, sorted, with exact counts.

    ``threads`` pieces with m-1 overlap (Sec. 2.6); 0 means one per host core.
    ``split_at`` (optional) fixes the threads-1 piece boundaries (window indices).
    Returns ``(locations uint32, mismatches uint32)``.
    """
    arr, n = _text_buf(text)
    pb = _pat(pattern)
    m = len(pb)
    if threads <= 0:
        threads = os.cpu_count() or 1
    split = None
    if split_at is not None:
        split = np.ascontiguousarray(np.asarray(split_at, dtype=np.uint64))
        threads = split.size + 1
    cap = 1 << 16
    while True:
        loc = np.empty(cap, dtype=np.uint32)
        mm = np.empty(cap, dtype=np.uint32)
        nh = ctypes.c_uint64(0)
        bad = ctypes.c_int64(-1)
        rc = lib().oracle_search(arr.ctypes.data, n, pb, m, int(k), 1 if early_exit else 0,
                                 threads, split.ctypes.data if split is not None else None,
                                 loc.ctypes.data, mm.ctypes.data, cap, ctypes.byref(nh),
                                 ctypes.byref(bad))
        if rc == E_OVERFLOW:
            cap = int(nh.value)
            continue
        if rc == E_SYMBOL:
            raise OracleError(f"text symbol outside Table 1 at offset {bad.value}")
        if rc != OK:
            raise OracleError(f"oracle_search failed: {rc}")
        h = int(nh.value)
        return loc[:h].copy(), mm[:h].copy()


def counts_unknown_text(text, pattern) -> np.ndarray:
    """Full sums for every window of a text that may hold symbols outside
    Table 1: such a symbol matches only the class N (see pm_oracle.c)."""
    arr, n = _text_buf(text)
    pb = _pat(pattern)
    m = len(pb)
    nwin = max(n - m + 1, 0)
    out = np.zeros(max(nwin, 1), dtype=np.uint32)
    rc = lib().oracle_counts_unknown_text(arr.ctypes.data, n, pb, m, out.ctypes.data)
    if rc != OK:
        raise OracleError(f"oracle_counts_unknown_text failed: {rc}")
    return out[:nwin]


def search_unknown_text(text, pattern, k: int) -> tuple[np.ndarray, np.ndarray]:
    """search() for a text that may hold symbols outside Table 1 (one
    thread): (locations uint32, mismatches uint32)."""
    arr, n = _text_buf(text)
    pb = _pat(pattern)
    cap = 1 << 16
    while True:
        loc = np.empty(cap, dtype=np.uint32)
        mm = np.empty(cap, dtype=np.uint32)
        nh = ctypes.c_uint64(0)
        rc = lib().oracle_search_unknown_text(arr.ctypes.data, n, pb, len(pb), int(k),
                                              loc.ctypes.data, mm.ctypes.data, cap, ctypes.byref(nh))
        if rc == E_OVERFLOW:
            cap = int(nh.value)
            continue
        if rc != OK:
            raise OracleError(f"oracle_search_unknown_text failed: {rc}")
        return loc[:nh.value].copy(), mm[:nh.value].copy()

