"""Pins for the oracle (CPU only).

Each test ties the oracle to something other than itself: the worked examples
printed in the paper (Sec. 1.1; Sec. 2.3; Sec. 2.5 with Table 4), the class
column of Table 2, the prime-product method of Sec. 1.3 (Eq. 1-3) computed in
exact integers, the numbers of Sec. 1.3.5, brute force over every short text,
and invariants of the definition (monotone in k, the Sec. 2.6 split with m-1
overlap, all-N and all-"-" patterns).
"""
import itertools
import json
import os

import numpy as np
import pytest

import oracle
from oracle import linhart_shamir as ls
from synth import IUPAC, random_pattern, uniform_text

GOLD = os.path.join(os.path.dirname(__file__), "golden")
SYMBOLS = "ACGTMRWSYKVHDBN-"


def golden(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def brute_counts(text: str, pattern: str) -> list[int]:
    """Definition of Sec. 1.1 with the classes of Table 2's class column."""
    return [sum(text[i + j] not in ls.CLASSES.get(pattern[j], "") for j in range(len(pattern)))
            for i in range(len(text) - len(pattern) + 1)]


# ------------------------------------------------ worked example, Sec. 2.5 --

def test_example2_codes():
    g = golden("example2_table4.json")
    assert [oracle.text_code(c) for c in g["text"]] == g["step1_text_codes"]
    assert [oracle.pattern_code(c) for c in g["pattern_iupac"]] == g["step2_pattern_codes"]
    r = [format(c << 2, "06b") for c in g["step2_pattern_codes"]]
    assert r == g["step3_r_binary"]


def test_example2_table4_trace():
    """Every index l and dictionary value of Table 4, and where each window stops at k = 2."""
    g = golden("example2_table4.json")
    for i1, lv in g["table4_l_values_at_k2"].items():
        got_l, got_v = oracle.window_trace(g["text"], g["pattern_iupac"], int(i1) - 1, k=g["k"])
        assert got_l == lv, f"window {i1}"
        assert got_v == g["table4_match_row_at_k2"][i1], f"window {i1}"


def test_example2_hits():
    g = golden("example2_table4.json")
    for k, key in ((0, "hits_k0"), (2, "hits_k2")):
        loc, mm = oracle.search(g["text"], g["pattern_iupac"], k)
        assert (loc + 1).tolist() == g[key]
        # a hit's count is the sum of its printed dictionary values
        for l1, c in zip((loc + 1).tolist(), mm.tolist()):
            assert c == sum(g["table4_match_row_at_k2"][str(l1)])


def test_sec2_3_examples():
    g = golden("example2_table4.json")["sec2_3_examples"]
    L = oracle.table3()
    A = oracle.text_code("A")
    assert L[oracle.lindex(oracle.pattern_code("M"), A)] == g["A_M"]
    assert L[oracle.lindex(oracle.pattern_code("B"), A)] == g["A_B"]
    assert oracle.lindex(oracle.pattern_code("D"), A) == g["A_D_index"]
    assert L[g["A_D_index"]] == g["A_D_value"]


# ------------------------------------------------ worked example, Sec. 1.1 --

def test_example1_sec1_1():
    g = golden("example1_sec1_1.json")
    # in the paper's own alphabet, by the definition t[i+j-1] in p[j]
    t, cls = g["text"], g["pattern_classes"]
    m = len(cls)
    mm = [sum(t[i + j] not in cls[j] for j in range(m)) for i in range(len(t) - m + 1)]
    assert [i + 1 for i, c in enumerate(mm) if c == 0] == g["hits_k0"]
    assert sorted(set(i + 1 for i, c in enumerate(mm) if c <= 2) - set(g["hits_k0"])) == \
        g["hits_k2_extra"]
    for i1, sub in g["substrings"].items():
        assert t[int(i1) - 1:int(i1) - 1 + m] == sub
    # the DNA reading through the oracle
    d = g["dna_reading"]
    assert "".join(d["map"][c] for c in t) == d["text"]
    loc, _ = oracle.search(d["text"], d["pattern_iupac"], 0)
    assert (loc + 1).tolist() == g["hits_k0"]
    loc, _ = oracle.search(d["text"], d["pattern_iupac"], 2)
    assert (loc + 1).tolist() == sorted(g["hits_k0"] + g["hits_k2_extra"])
    assert oracle.counts(d["text"], d["pattern_iupac"]).tolist() == mm


# --------------------------------------------------- Table 2 and Table 3 --

def test_table3_equals_table2_class_column():
    """L[(code(X) << 2) | code(a)] is 1 exactly when a is outside class X."""
    L = oracle.table3()
    for X in SYMBOLS:
        for a in "ACGT":
            l = oracle.lindex(oracle.pattern_code(X), oracle.text_code(a))
            assert L[l] == (a not in ls.CLASSES[X]), (X, a)
    assert sorted(oracle.pattern_code(X) for X in SYMBOLS) == list(range(16))


@pytest.mark.parametrize("primes", [[2, 3, 5, 7], ls.smallest_primes_above(1000),
                                    ls.smallest_primes_above(100_000)])
def test_table3_equals_prime_product(primes):
    """The per-pair residue test kept by the paper (Sec. 2, Eq. 1 and 3)."""
    L = oracle.table3()
    for X in SYMBOLS:
        for a in "ACGT":
            l = oracle.lindex(oracle.pattern_code(X), oracle.text_code(a))
            assert (L[l] == 0) == ls.pair_is_match(a, X, primes), (X, a, primes)


def test_unknown_pattern_symbols_are_dash():
    """Sec. 2.2: a missing or erroneous pattern symbol is coded 1111."""
    for ch in "XZ*?.1":
        assert oracle.pattern_code(ch) == 15
    assert oracle.count_unknown("ACXGZ") == 2
    assert oracle.count_unknown("acgtn-") == 0


# ----------------------------------------------------------- Sec. 1.3.5 --

def test_sec1_3_5_precision_numbers():
    g = golden("sec1_3_5_precision.json")
    primes = ls.smallest_primes_above(g["m"])
    assert primes == g["primes"]
    M = ls.modulus(primes)
    assert 0.5 * g["M_order"] < M < 5 * g["M_order"]
    for e in ls.text_codes(primes).values():
        assert 0.5 * g["e_order"] < e < 5 * g["e_order"]
    # a class code times a text code can leave uint64
    worst = max(ls.class_code(c, primes) for c in ls.CLASSES.values()) * max(ls.text_codes(primes).values())
    assert worst > 2 ** 64 > g["uint64_max_order"] / 2
    # for m = 1e5 the modulus alone no longer fits
    assert ls.modulus(ls.smallest_primes_above(100_000)) > 2 ** 64


# ------------------------------------ Linhart-Shamir route (Eq. 1-3) --

def test_crt_codes_satisfy_eq1():
    primes = ls.smallest_primes_above(7)
    for X, letters in ls.CLASSES.items():
        nS = ls.class_code(letters, primes)
        assert 0 <= nS < ls.modulus(primes)
        for a, q in zip("ACGT", primes):
            assert nS % q == (0 if a in letters else 1)


def test_oracle_equals_linhart_shamir_random_tiny():
    rng = np.random.default_rng(1234)
    for _ in range(60):
        n = int(rng.integers(1, 65))
        m = int(rng.integers(1, 9))
        t = "".join("ACGT"[x] for x in rng.integers(0, 4, n))
        p = "".join(SYMBOLS[x] for x in rng.integers(0, 16, m))
        if m > n:
            assert oracle.counts(t, p).size == 0
            continue
        assert oracle.counts(t, p).tolist() == ls.mismatch_counts(t, p)
        loc, _ = oracle.search(t, p, 0)
        assert loc.tolist() == ls.exact_locations(t, p)


# ------------------------------------------------------------ brute force --

@pytest.mark.parametrize("pattern", ["A", "N", "-", "CBG", "MRWSY", "KVHDBNA", "S-G"])
def test_exhaustive_texts_length7(pattern):
    """All 4^7 texts of length 7, against the definition with Table 2's classes."""
    m = len(pattern)
    texts = ["".join(x) for x in itertools.product("ACGT", repeat=7)]
    big = "".join(texts)
    full = oracle.counts(big, pattern)
    for q, t in enumerate(texts):
        expect = brute_counts(t, pattern)
        assert full[7 * q:7 * q + len(expect)].tolist() == expect, t


def test_random_against_definition():
    rng = np.random.default_rng(99)
    for _ in range(40):
        n = int(rng.integers(1, 300))
        m = int(rng.integers(1, 40))
        t = "".join("ACGT"[x] for x in rng.integers(0, 4, n))
        p = "".join(SYMBOLS[x] for x in rng.integers(0, 16, m))
        k = int(rng.integers(0, m + 2))
        full = brute_counts(t, p)
        loc, mm = oracle.search(t, p, k, threads=int(rng.integers(1, 6)))
        exp = [(i, c) for i, c in enumerate(full) if c <= k]
        assert list(zip(loc.tolist(), mm.tolist())) == exp


# -------------------------------------------------------------- invariants --

def test_early_exit_changes_nothing():
    rng = np.random.default_rng(5)
    t = uniform_text(20000, seed=5)
    for m in (1, 7, 32, 33, 100):
        p = random_pattern(m, m // 5, rng)
        for k in (0, 1, 3, m // 2, m):
            a = oracle.search(t, p, k, early_exit=True)
            b = oracle.search(t, p, k, early_exit=False)
            assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_monotone_in_k():
    rng = np.random.default_rng(6)
    t = uniform_text(30000, seed=6)
    p = random_pattern(24, 6, rng)
    prev = None
    for k in range(0, 26):
        loc, mm = oracle.search(t, p, k)
        cur = dict(zip(loc.tolist(), mm.tolist()))
        if prev is not None:
            assert all(cur.get(i) == c for i, c in prev.items())
        prev = cur
    assert len(prev) == 30000 - 24 + 1   # k >= m: every window


def test_k_at_least_m_reports_every_window():
    t = uniform_text(500, seed=8)
    for m in (1, 5, 17):
        loc, mm = oracle.search(t, ("MRWSYK" * 4)[:m], m)
        assert loc.tolist() == list(range(500 - m + 1))
        assert mm.max() <= m


def test_all_N_and_all_dash():
    t = uniform_text(1000, seed=9)
    assert oracle.counts(t, "N" * 13).tolist() == [0] * (1000 - 12)
    assert oracle.counts(t, "-" * 13).tolist() == [13] * (1000 - 12)
    assert oracle.counts(t, "Z" * 13).tolist() == [13] * (1000 - 12)


def test_split_with_overlap_any_point():
    """Sec. 2.6: pieces with m-1 overlap give the same hits wherever the cut is."""
    t = uniform_text(60, seed=10)
    p = "ACNGT"
    ref = oracle.search(t, p, 2, threads=1)
    nwin = 60 - 5 + 1
    for cut in range(0, nwin + 1):
        got = oracle.search(t, p, 2, split_at=[cut])
        assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])
    rng = np.random.default_rng(11)
    for _ in range(20):
        cuts = sorted(rng.integers(0, nwin + 1, size=int(rng.integers(1, 8))).tolist())
        got = oracle.search(t, p, 2, split_at=cuts)
        assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])
    for th in (1, 2, 3, 7, 64, 200):
        got = oracle.search(t, p, 2, threads=th)
        assert np.array_equal(got[0], ref[0])


def test_m_greater_than_n_and_bad_symbols():
    assert oracle.search("ACG", "ACGT", 5)[0].size == 0
    with pytest.raises(oracle.OracleError, match="offset 3"):
        oracle.search("ACGNACGT", "AC", 1)
    with pytest.raises(oracle.OracleError, match="offset 2"):
        oracle.search("AC#", "ACGT", 1)


def test_lowercase_is_uppercase():
    t = uniform_text(2000, seed=12)
    low = bytes(t).lower()
    p = "acgtmrwsykvhdbn-acgt"
    a = oracle.search(t, p.upper(), 8)
    b = oracle.search(low, p, 8)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_counts_at_matches_counts():
    t = uniform_text(5000, seed=13)
    p = "ACGTNNMRWS"
    full = oracle.counts(t, p)
    locs = np.array([0, 1, 17, 4989, 4990])
    assert oracle.counts_at(t, p, locs).tolist() == full[locs].tolist()


# ---- text symbols outside Table 1 (an extension; the reading is that an
# unknown text symbol matches the class N only) ----

def test_unknown_text_oracle_equals_table1_oracle_without_unknowns():
    rng = np.random.default_rng(500)
    for case in range(20):
        text = uniform_text(int(rng.integers(1, 400)), seed=500 + case)
        m = int(rng.integers(1, 20))
        pat = "".join(rng.choice(list("".join(IUPAC) + "-x"), size=m))
        assert np.array_equal(oracle.counts_unknown_text(text, pat), oracle.counts(text, pat))
        for k in (0, 2, 5):
            got = oracle.search_unknown_text(text, pat, k)
            want = oracle.search(text, pat, k, threads=1)
            assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])


def test_unknown_text_is_the_worst_letter_at_each_unknown():
    """With unknown symbols at a few offsets, every window's count equals the
    largest count over all ways of writing letters there: an unknown symbol
    mismatches every class but N, as the letter outside the class would."""
    rng = np.random.default_rng(501)
    for case in range(25):
        n = int(rng.integers(8, 60))
        text = uniform_text(n, seed=600 + case)
        u = int(rng.integers(1, 4))
        pos = rng.choice(n, size=u, replace=False)
        t_unk = text.copy()
        for q in pos:
            t_unk[q] = ord(rng.choice(list("NnRx*")))
        m = int(rng.integers(1, 9))
        pat = "".join(rng.choice(list("".join(IUPAC) + "-"), size=m))
        best = None
        for letters in itertools.product(b"ACGT", repeat=u):
            t = text.copy()
            t[pos] = letters
            c = oracle.counts(t, pat)
            best = c if best is None else np.maximum(best, c)
        assert np.array_equal(oracle.counts_unknown_text(t_unk, pat), best), (case, pat)


def test_unknown_text_all_unknown_and_search_consistency():
    text = np.frombuffer(b"N" * 50, dtype=np.uint8).copy()
    for pat in ("ACGT", "NNNN", "ANNT-", "RYKMSWBDHVN"):
        not_n = sum(1 for c in pat if c != "N")
        c = oracle.counts_unknown_text(text, pat)
        assert (c == not_n).all()
    rng = np.random.default_rng(502)
    text = uniform_text(3000, seed=502)
    text[rng.choice(3000, size=300, replace=False)] = ord("N")
    for m in (1, 7, 33):
        pat = random_pattern(m, m // 3, rng)
        full = oracle.counts_unknown_text(text, pat)
        for k in (0, 3, 10):
            loc, mm = oracle.search_unknown_text(text, pat, k)
            want = np.nonzero(full <= k)[0]
            assert np.array_equal(loc, want) and np.array_equal(mm, full[want])
