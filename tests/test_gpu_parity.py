"""Parity of the CUDA path (through the C ABI) with the oracle: bit-exact.

Every comparison is of sorted (location, mismatches) lists: integer work, so
the tolerance is zero.  Sizes span several 8192-window tiles with ragged
tails; pattern lengths straddle the 32-position chunk boundaries; k runs from
0 past m; both kernel variants are exercised.
"""
import json
import os

import numpy as np
import pytest

import oracle
import synth
from synth import workloads

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(__file__), "golden")
SYMBOLS = "ACGTMRWSYKVHDBN-"
# auto, pattern-sliced (32 positions), window-sliced, pattern-sliced (64
# positions), every chunk
VARIANTS = (0, 1, 2, 3, 4)


@pytest.fixture(scope="module")
def pm():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1611_06115_gb300 as pm
    pm.lib()  # fails loudly when libpm.so is missing: no fallback
    return pm


def gpu_hits(pm, text, patterns, ks, variant=0, out="device", capacity=None):
    t = pm.pm_encode_text(text)
    pats = [pm.pm_compile_pattern(p) for p in patterns]
    r = pm.pm_search_ex(t, pats, ks, capacity=capacity, out=out, variant=variant)
    return [r.pattern(i) for i in range(len(pats))]


def same(got, exp):
    gl, gm = got
    el, em = exp
    assert gl.dtype == np.uint32 and gm.dtype == np.uint32
    assert np.array_equal(gl, el), (gl[:10], el[:10], gl.size, el.size)
    assert np.array_equal(gm, em)


def test_worked_example_sec2_5(pm):
    with open(os.path.join(GOLD, "example2_table4.json")) as f:
        g = json.load(f)
    for v in VARIANTS:
        (l0, m0), (l2, m2) = gpu_hits(pm, g["text"], [g["pattern_iupac"]] * 2, [0, 2], variant=v)
        assert (l0 + 1).tolist() == g["hits_k0"] and m0.tolist() == [0]
        assert (l2 + 1).tolist() == g["hits_k2"]
        for l1, c in zip((l2 + 1).tolist(), m2.tolist()):
            assert c == sum(g["table4_match_row_at_k2"][str(l1)])


def test_worked_example_sec1_1(pm):
    with open(os.path.join(GOLD, "example1_sec1_1.json")) as f:
        g = json.load(f)
    d = g["dna_reading"]
    (l0, _), (l2, _) = gpu_hits(pm, d["text"], [d["pattern_iupac"]] * 2, [0, 2])
    assert (l0 + 1).tolist() == g["hits_k0"]
    assert (l2 + 1).tolist() == sorted(g["hits_k0"] + g["hits_k2_extra"])


@pytest.mark.parametrize("variant", VARIANTS)
def test_random_small_against_oracle(pm, variant):
    rng = np.random.default_rng(100 + variant)
    for case in range(30):
        n = int(rng.integers(1, 60000))
        m = int(rng.choice([1, 2, 5, 17, 31, 32, 33, 63, 64, 65, 100, 257, 1000, 3000]))
        k = int(rng.choice([0, 1, 2, 3, 5, 8, 16, 31, 32, max(m // 2, 0), m, m + 1]))
        text = synth.uniform_text(n, seed=case)
        # mostly plain letters with some classes, N, "-" and unknown bytes
        alphabet = "ACGT" * 6 + SYMBOLS + "xz"
        pat = "".join(alphabet[i] for i in rng.integers(0, len(alphabet), m))
        exp = oracle.search(text, pat, k)
        got = gpu_hits(pm, text, [pat], [k], variant=variant)[0]
        same(got, exp)


def test_planted_copies_many_tiles_ragged(pm):
    rng = np.random.default_rng(7)
    n = 5 * 8192 * 4 + 777
    text = synth.markov_text(n, seed=9)
    pats = [synth.random_pattern(m, m // 10, rng) for m in (32, 33, 96, 500)]
    occ = synth.Occupancy()
    planted = [synth.plant(text, p, 30, 6, rng, occ) for p in pats]
    ks = [6, 6, 6, 6]
    for v in VARIANTS:
        got = gpu_hits(pm, text, pats, ks, variant=v)
        for p, pl, g in zip(pats, planted, got):
            same(g, oracle.search(text, p, 6))
            found = dict(zip(g[0].tolist(), g[1].tolist()))
            for loc, s in pl:
                assert found.get(loc) == s


@pytest.mark.parametrize("variant", VARIANTS)
def test_dense_hits_every_window(pm, variant):
    n = 3 * 8192 + 4321
    text = synth.uniform_text(n, seed=3)
    for m, k in ((1, 1), (40, 40), (70, 100)):
        pat = ("MRWSYKVHDB" * 10)[:m]
        l, c = gpu_hits(pm, text, [pat], [k], variant=variant)[0]
        assert l.tolist() == list(range(n - m + 1))
        assert np.array_equal(c, oracle.counts(text, pat))


@pytest.mark.parametrize("variant", VARIANTS)
def test_edges_m_vs_n(pm, variant):
    text = synth.uniform_text(100, seed=4)
    (l, _), = gpu_hits(pm, text, ["A" * 101], [200], variant=variant)
    assert l.size == 0
    (l, c), = gpu_hits(pm, text, [bytes(text).decode()], [0], variant=variant)
    assert l.tolist() == [0] and c.tolist() == [0]
    for k in (0, 3, 6):  # one window per tile edge region: n = 4096*32*j + r
        t2 = synth.uniform_text(4096 * 32 + 33, seed=40 + k)
        pat = bytes(t2[4096 * 32 - 5:4096 * 32 + 27]).decode()  # straddles the first tile boundary
        (l, c), = gpu_hits(pm, t2, [pat], [k], variant=variant)
        same((l, c), oracle.search(t2, pat, k))
    t0 = pm.pm_encode_text(b"")
    r = pm.pm_search(t0, [pm.pm_compile_pattern("ACG")], [1])
    assert r.total == 0 and r.offsets.cpu().tolist() == [0, 0]
    r = pm.pm_search(t0, [], [])
    assert r.offsets.cpu().tolist() == [0]


def test_all_N_all_dash_unknown(pm):
    text = synth.uniform_text(20000, seed=5)
    (ln, cn), (ld, cd), (lu, cu) = gpu_hits(pm, text, ["N" * 45, "-" * 45, "#" * 45],
                                             [0, 45, 44])
    assert ln.size == 20000 - 44 and not cn.any()
    assert ld.size == 20000 - 44 and (cd == 45).all()
    assert lu.size == 0


def test_overflow_then_exact_capacity(pm):
    text = synth.uniform_text(30000, seed=6)
    t = pm.pm_encode_text(text)
    p = pm.pm_compile_pattern("ACGTNN")
    exp = oracle.search(text, "ACGTNN", 2)
    with pytest.raises(pm.PmError) as e:
        pm.pm_search_ex(t, [p], [2], capacity=10)
    assert e.value.status == pm.PM_E_OVERFLOW
    r = pm.pm_search_ex(t, [p], [2], capacity=exp[0].size)
    same(r.pattern(0), exp)
    r = pm.pm_search_ex(t, [p], [2])  # grows on overflow
    same(r.pattern(0), exp)


def test_host_and_device_outputs_and_async(pm):
    import torch
    text = synth.markov_text(70000, seed=8)
    pats = ["ACGTRYN", "CCCCGGGGAAAATTTTMMKK", "W" * 40]
    ks = [1, 5, 10]
    a = gpu_hits(pm, text, pats, ks, out="device")
    b = gpu_hits(pm, text, pats, ks, out="host")
    for x, y, p, k in zip(a, b, pats, ks):
        same(x, y)
        same(x, oracle.search(text, p, k))
    t = pm.pm_encode_text(text)
    cp = [pm.pm_compile_pattern(p) for p in pats]
    r = pm.pm_search_ex(t, cp, ks, capacity=1 << 16, sync=False)
    torch.cuda.synchronize()
    for i, (p, k) in enumerate(zip(pats, ks)):
        same(r.pattern(i), oracle.search(text, p, k))


def test_repeated_handles_varied_k_monotone(pm):
    text = synth.markov_text(100000, seed=10)
    pat = synth.random_pattern(48, 5, np.random.default_rng(1))
    t = pm.pm_encode_text(text)
    p = pm.pm_compile_pattern(pat)
    ks = list(range(0, 20))
    r = pm.pm_search(t, [p] * len(ks), ks)
    prev = {}
    for i, k in enumerate(ks):
        l, c = r.pattern(i)
        same((l, c), oracle.search(text, pat, k))
        cur = dict(zip(l.tolist(), c.tolist()))
        assert all(cur.get(x) == y for x, y in prev.items())
        prev = cur


def test_text_coding_errors_and_case(pm):
    with pytest.raises(pm.PmError) as e:
        pm.pm_encode_text(b"ACGTACGTNACGT")
    assert e.value.status == pm.PM_E_SYMBOL and "offset 8" in str(e.value)
    with pytest.raises(pm.PmError) as e:
        pm.pm_encode_text(b"A" * 100 + b"\x00")
    assert "offset 100" in str(e.value)
    text = synth.uniform_text(5000, seed=11)
    low = np.frombuffer(bytes(text).lower(), dtype=np.uint8)
    a = gpu_hits(pm, text, ["ACGTMK"], [2])[0]
    b = gpu_hits(pm, low, ["acgtmk"], [2])[0]
    same(a, b)


def test_device_resident_ascii_input(pm):
    import torch
    text = synth.uniform_text(123457, seed=12)
    d = torch.from_numpy(text).cuda()
    t = pm.pm_encode_text(d)
    p = pm.pm_compile_pattern("GATTACA")
    same(pm.pm_search(t, [p], [1]).pattern(0), oracle.search(text, "GATTACA", 1))
    # an unaligned device pointer takes the byte path
    t2 = pm.pm_encode_text(d[3:])
    same(pm.pm_search(t2, [p], [1]).pattern(0), oracle.search(text[3:], "GATTACA", 1))


def test_pr1_workload(pm):
    """PR1: n = 1e6 uniform text, m = 16 with 4 class positions, 20 planted
    copies with 0-3 substitutions, k in {0, 2}; sorted int32 pairs."""
    w = workloads.pr1()
    pat = w.patterns[0]
    for v in VARIANTS:
        got = gpu_hits(pm, w.text, [pat, pat], [0, 2], variant=v)
        for (l, c), k in zip(got, (0, 2)):
            same((l, c), oracle.search(w.text, pat, k))
            pairs = np.stack([l, c], axis=1).astype(np.int32)
            assert (np.diff(pairs[:, 0]) > 0).all()
            found = dict(zip(l.tolist(), c.tolist()))
            for loc, s in w.planted[0]:
                if s <= k:
                    assert found.get(loc) == s


def test_genome_recipe_reduced(pm):
    """The GENOME recipe (Markov text, m in {32, 128, 1024}, k in {0, 4, 16},
    planted copies) at n = 3e7, checked window for window."""
    w = workloads.genome(n=30_000_000, copies=40)
    pats, ks = [], []
    for p in w.patterns:
        for k in (0, 4, 16):
            pats.append(p)
            ks.append(k)
    got = gpu_hits(pm, w.text, pats, ks)
    for (l, c), p, k in zip(got, pats, ks):
        same((l, c), oracle.search(w.text, p, k))
    for pi, pl in enumerate(w.planted):
        for kk, k in enumerate((0, 4, 16)):
            found = dict(zip(*[a.tolist() for a in got[3 * pi + kk]]))
            for loc, s in pl:
                if s <= k:
                    assert found.get(loc) == s


def test_large_patterns_reduced(pm):
    """The LARGE recipe (m in {1e4, 1e5}, 5 % classes, k in {0, 100, 1000})
    at n = 1.5e6: long patterns, many chunks per window."""
    w = workloads.large(n=1_500_000, copies=4)
    for p in w.patterns:
        got = gpu_hits(pm, w.text, [p] * 3, [0, 100, 1000])
        for (l, c), k in zip(got, (0, 100, 1000)):
            same((l, c), oracle.search(w.text, p, k))


@pytest.mark.parametrize("variant", (1, 3, 4))
def test_mid_k_many_survivors(pm, variant):
    """k from 17 to 63 on patterns of two to ten chunks: many windows survive
    the first 32 (or 64) positions and are settled one by one, or counted by
    every chunk; all forms give the oracle's hits."""
    rng = np.random.default_rng(40 + variant)
    n = 3 * 4096 * 32 + 321
    text = synth.markov_text(n, seed=31)
    pats, ks = [], []
    for m in (40, 64, 65, 96, 130, 300):
        for k in (17, 20, 24, 31, 40, 63):
            pats.append(synth.random_pattern(m, m // 10, rng))
            ks.append(k)
    got = gpu_hits(pm, text, pats, ks, variant=variant)
    for p, k, g in zip(pats, ks, got):
        same(g, oracle.search(text, p, k))


def test_auto_variant_table(pm):
    """pm_set_auto_variants: any valid table gives the same hits; invalid
    tables are rejected and leave the table unchanged; [] restores it."""
    rng = np.random.default_rng(77)
    text = synth.markov_text(2 * 4096 * 32 + 55, seed=8)
    pats = [synth.random_pattern(m, m // 10, rng) for m in (20, 70, 200)]
    ks = [0, 5, 18, 33]
    exp = [[oracle.search(text, p, k) for k in ks] for p in pats]
    builtin = pm.pm_get_auto_variants()
    assert len(builtin) == 64
    tables = ([pm.PM_VARIANT_ALL_CHUNKS] * 64,
              [pm.PM_VARIANT_WINDOW_SLICED if k <= 8 else pm.PM_VARIANT_PATTERN_SLICED_2 for k in range(64)],
              [pm.PM_VARIANT_PATTERN_SLICED] * 20)
    try:
        for table in tables:
            pm.pm_set_auto_variants(table)
            assert pm.pm_get_auto_variants(len(table)) == list(table)
            for p, e in zip(pats, exp):
                got = gpu_hits(pm, text, [p] * len(ks), ks)
                for g, x in zip(got, e):
                    same(g, x)
        before = pm.pm_get_auto_variants()
        for bad in ([pm.PM_VARIANT_AUTO], [pm.PM_VARIANT_WINDOW_SLICED] * 10, [pm.PM_VARIANT_PATTERN_SLICED] * 33,
                    [7], [pm.PM_VARIANT_ALL_CHUNKS] * 65):
            with pytest.raises(pm.PmError):
                pm.pm_set_auto_variants(bad)
            assert pm.pm_get_auto_variants() == before
    finally:
        pm.pm_set_auto_variants([])
    assert pm.pm_get_auto_variants() == builtin



def test_letter_counts_and_position_order(pm):
    """pm_text_letter_counts equals a count of the ASCII text (host and device
    input, ragged length, lower case); a text rich in one letter reorders the
    window-sliced positions, which leaves every hit as the oracle has it."""
    import torch
    rng = np.random.default_rng(90)
    for n in (1, 31, 4096 * 32 * 2 + 77):
        text = synth.markov_text(n, seed=n)
        want = [int(np.count_nonzero(text == ord(c))) for c in "ACGT"]
        assert pm.pm_encode_text(text).letter_counts() == want
        low = text.copy()
        low[::3] |= 0x20
        assert pm.pm_encode_text(torch.from_numpy(low).cuda()).letter_counts() == want
    # 85 % T: positions asking for T are tested last, the rest first
    n = 3 * 4096 * 32 + 5
    text = np.frombuffer(np.where(rng.random(n) < 0.85, ord("T"),
                                  rng.choice(np.frombuffer(b"ACG", np.uint8), n)).astype(np.uint8).tobytes(),
                         np.uint8).copy()
    pats = ["TTTTATTTTCTTTTGTTTTTRTTTYTTTTTTT" + "TTATT", "ACGTTTTTACGTTTTT", "TTTTTTTTTTTTTTTTTTTTTTTTTTTTTTTTTTTT"]
    for v in (0, 2):
        for k in (0, 1, 2, 4):
            got = gpu_hits(pm, text, pats, [k] * 3, variant=v)
            for p, g in zip(pats, got):
                same(g, oracle.search(text, p, k))


def test_text_save_and_load(pm, tmp_path):
    """A coded text written to a file and read back searches the same; a
    corrupted or foreign file is refused."""
    rng = np.random.default_rng(91)
    text = synth.markov_text(2 * 4096 * 32 + 71, seed=91)
    unk = text.copy()
    unk[5000:5400] = ord("N")
    pats = [synth.random_pattern(m, m // 10, rng) for m in (20, 64, 300)]
    for src, flags in ((text, 0), (unk, pm.PM_TEXT_UNKNOWN_AS_N)):
        t = pm.pm_encode_text_ex(src, flags=flags)
        path = str(tmp_path / f"t{flags}.pmtext")
        t.save(path)
        back = pm.Text.load(path)
        assert back.n == t.n and back.unknown() == t.unknown()
        assert back.letter_counts() == t.letter_counts()
        cps = [pm.pm_compile_pattern(p) for p in pats]
        a = pm.pm_search(t, cps, [0, 3, 12])
        b = pm.pm_search(back, cps, [0, 3, 12])
        assert np.array_equal(a.numpy()[0], b.numpy()[0]) and np.array_equal(a.numpy()[1], b.numpy()[1])
        for i, (p, k) in enumerate(zip(pats, (0, 3, 12))):
            exp = oracle.search_unknown_text(src, p, k) if flags else oracle.search(src, p, k)
            same(b.pattern(i), exp)
        raw = bytearray(open(path, "rb").read())
        raw[-100] ^= 0x40
        bad = str(tmp_path / "bad.pmtext")
        open(bad, "wb").write(bytes(raw))
        with pytest.raises(pm.PmError) as e:
            pm.Text.load(bad)
        assert e.value.status == pm.PM_E_ARG
    foreign = str(tmp_path / "foreign")
    open(foreign, "wb").write(b"ACGT" * 100)
    with pytest.raises(pm.PmError):
        pm.Text.load(foreign)


@pytest.mark.parametrize("k", range(0, 9))
def test_window_sliced_every_k(pm, k):
    """The window-sliced evaluation at every k it takes (a thermometer counter
    below k = 4, carry-save binary counters from k = 4 on), forced for
    patterns of one to many chunks, with class-heavy first chunks (class
    positions go through the counters four at a time, runs of one letter
    end partway through a block of four), over a text of several 8192-window
    tiles with a ragged tail; element by element against the oracle."""
    rng = np.random.default_rng(100 + k)
    text = synth.markov_text(3 * 8192 * 32 + 777, seed=20 + k)
    t = pm.pm_encode_text(text)
    pats = [synth.random_pattern(m, nc, rng) for m, nc in ((9, 1), (17, 9), (32, 3), (45, 20), (130, 13))]
    cps = [pm.pm_compile_pattern(p) for p in pats]
    r = pm.pm_search_ex(t, cps, [k] * len(cps), variant=pm.PM_VARIANT_WINDOW_SLICED)
    for i, p in enumerate(pats):
        same(r.pattern(i), oracle.search(text, p, k))
