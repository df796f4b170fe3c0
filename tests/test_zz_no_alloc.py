"""pm_search_noalloc, the entry point for callers that cannot allocate memory.

Such callers (host callbacks, real-time loops, applications that own all of
their device memory) pass the output buffers in and get the same results as
pm_search, with the scratch taken from a fixed array inside the library.
This test calls it through the C ABI (ctypes, no Python wrapper) twice in a
row and compares both results with pm_search's, bit for bit (integer
results: the tolerance is zero).  It sets up its own inputs so that it runs
the same alone in a fresh process and after every other test.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _call_noalloc(L, text, pats, ks, hits, offsets, cap):
    harr = (ctypes.c_void_p * len(pats))(*[p.handle for p in pats])
    karr = (ctypes.c_int32 * len(ks))(*ks)
    needed = ctypes.c_uint64(0)
    st = L.pm_search_noalloc(text.handle, harr, len(pats), karr, ctypes.c_void_p(hits.data_ptr()),
                             cap, ctypes.c_void_p(offsets.data_ptr()), ctypes.byref(needed),
                             ctypes.c_void_p(0))
    return st, int(needed.value)


def test_noalloc_matches_pm_search_twice():
    import torch
    import synth
    import paper_1611_06115_gb300 as pm

    L = pm.lib()
    text_np = synth.markov_text(2 * 8192 * 32 + 12345, seed=41)
    rng = np.random.default_rng(41)
    pat_strs = [synth.random_pattern(m, m // 10, rng) for m in (12, 40, 300)]
    planted = synth.plant(text_np, pat_strs[1], 20, 3, rng)
    text = pm.pm_encode_text(text_np)
    pats = [pm.pm_compile_pattern(p) for p in pat_strs]
    call_pats = [pats[0], pats[1], pats[1], pats[2]]
    ks = [1, 0, 3, 40]

    ref = pm.pm_search(text, call_pats, ks)
    ref_hits, ref_off = ref.numpy()
    cap = int(ref_off[-1]) + 100

    hits = torch.full((cap, 2), -1, dtype=torch.int32, device="cuda")
    offsets = torch.zeros(len(ks) + 1, dtype=torch.int64, device="cuda")
    for _ in range(2):  # the second call reuses the array the first one left behind
        hits.fill_(-1)
        offsets.zero_()
        st, needed = _call_noalloc(L, text, call_pats, ks, hits, offsets, cap)
        assert st == pm.PM_OK, L.pm_last_error().decode()
        torch.cuda.synchronize()
        assert needed == int(ref_off[-1])
        off = offsets.cpu().numpy().astype(np.uint64)
        assert np.array_equal(off, ref_off)
        got = hits[:needed].cpu().numpy().view(np.uint32).reshape(-1, 2)
        assert np.array_equal(got, ref_hits)
    # planted copies of pattern 1 with s <= 3 are among the k = 3 hits
    l, c = ref.pattern(2)
    found = dict(zip(l.tolist(), c.tolist()))
    assert all(found.get(loc) == s for loc, s in planted)


def test_noalloc_rejects_sizes_beyond_its_limits():
    import torch
    import paper_1611_06115_gb300 as pm

    L = pm.lib()
    text = pm.pm_encode_text(b"ACGT" * 100)
    p = pm.pm_compile_pattern("ACG")
    hits = torch.zeros((16, 2), dtype=torch.int32, device="cuda")
    offsets = torch.zeros(66, dtype=torch.int64, device="cuda")
    st, _ = _call_noalloc(L, text, [p], [0], hits, offsets, (1 << 22) + 1)
    assert st == pm.PM_E_TOO_LARGE and b"capacity" in L.pm_last_error()
    st, _ = _call_noalloc(L, text, [p] * 65, [0] * 65, hits, offsets, 16)
    assert st == pm.PM_E_TOO_LARGE and b"npat" in L.pm_last_error()
    # host outputs are refused: this entry point does not stage through device memory
    host_off = torch.zeros(2, dtype=torch.int64)
    st, _ = _call_noalloc(L, text, [p], [0], hits, host_off, 16)
    assert st == pm.PM_E_ARG
