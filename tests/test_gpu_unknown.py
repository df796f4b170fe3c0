"""Texts with symbols outside Table 1 (pm_encode_text_ex, PM_TEXT_UNKNOWN_AS_N):
an unknown symbol matches the class N only.  Every evaluation, the batched
launch and the no-allocation entry point give the oracle's hits, bit for
bit."""
import ctypes

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pm():
    import torch
    assert torch.cuda.is_available()
    import paper_1611_06115_gb300 as pm
    pm.lib()
    return pm


def text_with_unknowns(n, seed):
    """Markov text with N runs (1 .. 5000 long), scattered single unknown
    bytes of several kinds, and lower case."""
    rng = np.random.default_rng(seed)
    t = synth.markov_text(n, seed=seed)
    for _ in range(12):
        a = int(rng.integers(0, n))
        t[a:a + int(rng.integers(1, 5000))] = ord("N")
    pos = rng.choice(n, size=n // 500, replace=False)
    t[pos] = rng.choice(np.frombuffer(b"NnRYx-*", np.uint8), size=pos.size)
    low = rng.choice(n, size=n // 7, replace=False)
    t[low] |= np.where(np.isin(t[low], np.frombuffer(b"ACGT", np.uint8)), 0x20, 0).astype(np.uint8)
    return t


def patterns(rng):
    out = []
    for m in (1, 5, 31, 32, 33, 64, 100, 500):
        out.append(synth.random_pattern(m, m // 8, rng))
    out.append("N" * 20)
    out.append("ANNNNNNT")
    out.append("A" * 40)  # all of an N run codes as some letter: every window there is a candidate
    out.append("-" * 3 + "ACGT")
    return out


def hits(res, i):
    l, c = res.pattern(i)
    return l, c


def test_counts_and_strict_coding(pm):
    t = text_with_unknowns(50_000, 3)
    with pytest.raises(pm.PmError) as e:
        pm.pm_encode_text(t)
    assert e.value.status == pm.PM_E_SYMBOL
    with pytest.raises(pm.PmError) as e:
        pm.pm_encode_text_ex(t, flags=2)
    assert e.value.status == pm.PM_E_ARG
    tx = pm.pm_encode_text_ex(t, flags=pm.PM_TEXT_UNKNOWN_AS_N)
    up = t & 0xDF
    unknown = int(np.count_nonzero(~np.isin(up, np.frombuffer(b"ACGT", np.uint8))))
    assert tx.unknown() == unknown
    assert tx.letter_counts() == [int(np.count_nonzero(up == ord(c))) for c in "ACGT"]
    # the flag on a text without unknown symbols changes nothing
    clean = synth.markov_text(10_000, seed=4)
    a = pm.pm_encode_text_ex(clean, flags=pm.PM_TEXT_UNKNOWN_AS_N)
    assert a.unknown() == 0
    assert a.letter_counts() == pm.pm_encode_text(clean).letter_counts()


@pytest.mark.parametrize("variant", (0, 1, 2, 3, 4))
def test_search_matches_oracle(pm, variant):
    import torch
    rng = np.random.default_rng(10 + variant)
    n = 3 * 4096 * 32 + 1234
    t = text_with_unknowns(n, 20 + variant)
    tx = pm.pm_encode_text_ex(torch.from_numpy(t).cuda() if variant == 2 else t,
                              flags=pm.PM_TEXT_UNKNOWN_AS_N)
    pats = patterns(rng)
    for ks in ((0,) * len(pats), (2,) * len(pats), tuple(min(len(p), 1 + len(p) // 4) for p in pats)):
        cps = [pm.pm_compile_pattern(p) for p in pats]
        res = pm.pm_search_ex(tx, cps, list(ks), variant=variant)
        for i, (p, k) in enumerate(zip(pats, ks)):
            el, em = oracle.search_unknown_text(t, p, k)
            gl, gm = hits(res, i)
            assert np.array_equal(gl, el), (p[:20], k, gl[:5], el[:5])
            assert np.array_equal(gm, em), (p[:20], k)


def test_batch_and_noalloc_match_oracle(pm):
    import torch
    rng = np.random.default_rng(30)
    n = 2 * 4096 * 32 + 77
    t = text_with_unknowns(n, 31)
    tx = pm.pm_encode_text_ex(t, flags=pm.PM_TEXT_UNKNOWN_AS_N)
    pats = patterns(rng)
    ks = [int(rng.integers(0, 1 + len(p) // 3)) for p in pats]
    cps = [pm.pm_compile_pattern(p) for p in pats]
    ref = pm.pm_search(tx, cps, ks)
    for i, (p, k) in enumerate(zip(pats, ks)):
        el, em = oracle.search_unknown_text(t, p, k)
        gl, gm = hits(ref, i)
        assert np.array_equal(gl, el) and np.array_equal(gm, em), (p[:20], k)
    b = pm.Batch(tx, cps, ks, capacity=ref.total + 8)
    out = b.run()
    torch.cuda.synchronize()
    assert out.total == ref.total
    assert np.array_equal(out.numpy()[0], ref.numpy()[0])
    assert np.array_equal(out.numpy()[1], ref.numpy()[1])
    # the entry point that allocates nothing
    L = pm.lib()
    cap = ref.total + 8
    h = torch.empty((cap, 2), dtype=torch.int32, device="cuda")
    off = torch.empty(len(cps) + 1, dtype=torch.int64, device="cuda")
    harr = (ctypes.c_void_p * len(cps))(*[c.handle for c in cps])
    karr = (ctypes.c_int32 * len(ks))(*ks)
    needed = ctypes.c_uint64(0)
    st = L.pm_search_noalloc(tx.handle, harr, len(cps), karr, ctypes.c_void_p(h.data_ptr()), cap,
                             ctypes.c_void_p(off.data_ptr()), ctypes.byref(needed), ctypes.c_void_p(0))
    assert st == 0 and needed.value == ref.total
    torch.cuda.synchronize()
    assert np.array_equal(off.cpu().numpy(), ref.offsets.cpu().numpy())
    assert np.array_equal(h[:ref.total].cpu().numpy(), ref.hits[:ref.total].cpu().numpy())
