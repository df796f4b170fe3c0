"""pm_search_noalloc, the entry point for callers that cannot allocate memory.

Such callers (real-time loops that may not take the allocator's locks or
its synchronisation, applications that own all of their device memory) pass
the output buffers in and get the same results as pm_search, with the
scratch taken from a fixed array inside the library.
This test calls it through the C ABI (ctypes, no Python wrapper) twice in a
row and compares both results with pm_search's, bit for bit (integer
results: the tolerance is zero).  It sets up its own inputs so that it runs
the same alone in a fresh process and after every other test.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _call_noalloc(L, text, pats, ks, hits, offsets, cap, want_needed=True):
    harr = (ctypes.c_void_p * len(pats))(*[p.handle for p in pats])
    karr = (ctypes.c_int32 * len(ks))(*ks)
    needed = ctypes.c_uint64(0)
    st = L.pm_search_noalloc(text.handle, harr, len(pats), karr, ctypes.c_void_p(hits.data_ptr()),
                             cap, ctypes.c_void_p(offsets.data_ptr()),
                             ctypes.byref(needed) if want_needed else None, ctypes.c_void_p(0))
    return st, int(needed.value)


# CUDA driver API through ctypes (the driver library is present wherever a
# GPU is): the device's default stream-ordered memory pool and its free memory
_CU_MEMPOOL_ATTR_RESERVED_MEM_HIGH = 6
_CU_MEMPOOL_ATTR_USED_MEM_HIGH = 8


def _cu():
    cu = ctypes.CDLL("libcuda.so.1")
    cu.cuDeviceGetDefaultMemPool.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int]
    cu.cuMemPoolGetAttribute.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
    cu.cuMemPoolSetAttribute.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
    cu.cuMemGetInfo_v2.argtypes = [ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_size_t)]
    return cu


def _pool(cu):
    import torch
    pool = ctypes.c_void_p()
    assert cu.cuDeviceGetDefaultMemPool(ctypes.byref(pool), torch.cuda.current_device()) == 0
    return pool


def _reset_pool_marks():
    """Reset the high-water marks of the device's default memory pool."""
    cu = _cu()
    pool = _pool(cu)
    zero = ctypes.c_uint64(0)
    for attr in (_CU_MEMPOOL_ATTR_RESERVED_MEM_HIGH, _CU_MEMPOOL_ATTR_USED_MEM_HIGH):
        assert cu.cuMemPoolSetAttribute(pool, attr, ctypes.byref(zero)) == 0


def _device_memory_marks():
    """(free device bytes, reserved high-water mark, used high-water mark of
    the default memory pool) of the current device."""
    cu = _cu()
    pool = _pool(cu)
    marks = []
    for attr in (_CU_MEMPOOL_ATTR_RESERVED_MEM_HIGH, _CU_MEMPOOL_ATTR_USED_MEM_HIGH):
        v = ctypes.c_uint64(0)
        assert cu.cuMemPoolGetAttribute(pool, attr, ctypes.byref(v)) == 0
        marks.append(int(v.value))
    free, total = ctypes.c_size_t(0), ctypes.c_size_t(0)
    assert cu.cuMemGetInfo_v2(ctypes.byref(free), ctypes.byref(total)) == 0
    return int(free.value), marks[0], marks[1]


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
    # the entry point's first call on this device looks up its array
    st, _ = _call_noalloc(L, text, call_pats, ks, hits, offsets, cap)
    assert st == pm.PM_OK, L.pm_last_error().decode()
    torch.cuda.synchronize()
    _reset_pool_marks()
    before = _device_memory_marks()
    for _ in range(2):  # the second call reuses the array the first one left behind
        hits.fill_(-1)
        offsets.zero_()
        torch.cuda.synchronize()
        st, needed = _call_noalloc(L, text, call_pats, ks, hits, offsets, cap)
        assert st == pm.PM_OK, L.pm_last_error().decode()
        torch.cuda.synchronize()
        # no allocation: neither the stream-ordered pool nor the device's free memory moved
        free, reserved_high, used_high = _device_memory_marks()
        assert reserved_high == before[1] and used_high == before[2], (before, reserved_high, used_high)
        assert free == before[0]
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


def test_noalloc_overflow_and_missing_needed():
    """An output that does not fit: PM_E_OVERFLOW with *needed the true count
    and no hit written; without `needed` the call returns at once and
    offsets[npat] carries the total (the array's leftovers from earlier calls
    must not leak into either)."""
    import torch
    import synth
    import paper_1611_06115_gb300 as pm

    L = pm.lib()
    text_np = synth.markov_text(3 * 8192 * 32 + 555, seed=44)
    text = pm.pm_encode_text(text_np)
    p = pm.pm_compile_pattern("ACGTN")  # many hits at k = 2
    ref = pm.pm_search(text, [p], [2])
    total = ref.total
    assert total > 200
    hits = torch.full((total, 2), -5, dtype=torch.int32, device="cuda")
    offsets = torch.zeros(2, dtype=torch.int64, device="cuda")
    small = total // 2
    st, needed = _call_noalloc(L, text, [p], [2], hits, offsets, small)
    assert st == pm.PM_E_OVERFLOW and needed == total
    torch.cuda.synchronize()
    assert int(offsets[-1].item()) == total
    assert bool((hits == -5).all().item())  # nothing written when the output does not fit
    # needed = NULL: asynchronous, the total lands in offsets[npat]
    offsets.zero_()
    st, _ = _call_noalloc(L, text, [p], [2], hits, offsets, total, want_needed=False)
    assert st == pm.PM_OK
    torch.cuda.synchronize()
    assert int(offsets[-1].item()) == total
    got = hits[:total].cpu().numpy().view(np.uint32).reshape(-1, 2)
    assert np.array_equal(got, ref.numpy()[0])


def test_noalloc_chunk_and_tile_limits():
    """Beyond 4096 pattern chunks or 2^21 warp tiles: PM_E_TOO_LARGE with
    nothing queued."""
    import torch
    import synth
    import paper_1611_06115_gb300 as pm

    L = pm.lib()
    hits = torch.zeros((16, 2), dtype=torch.int32, device="cuda")
    offsets = torch.zeros(66, dtype=torch.int64, device="cuda")
    small = pm.pm_encode_text(b"ACGT" * 1000)
    long_pat = pm.pm_compile_pattern("A" * (4096 * 32 + 1))  # 4097 chunks
    st, _ = _call_noalloc(L, small, [long_pat], [0], hits, offsets, 16)
    assert st == pm.PM_E_TOO_LARGE and b"chunks" in L.pm_last_error()
    # 64 pairs at k = 12 (pattern-sliced: tiles of 4096 windows) over 140e6
    # symbols: 64 x 34180 > 2^21 tiles
    big = pm.pm_encode_text(synth.markov_text(140_000_000, seed=45))
    p = pm.pm_compile_pattern("ACGTACGTAC" * 3 + "AC")
    st, _ = _call_noalloc(L, big, [p] * 64, [12] * 64, hits, offsets, 16)
    assert st == pm.PM_E_TOO_LARGE and b"tiles" in L.pm_last_error()
    # the same search within the limit (fewer pairs) runs
    st, needed = _call_noalloc(L, big, [p] * 8, [12] * 8, hits, offsets, 16)
    assert st in (pm.PM_OK, pm.PM_E_OVERFLOW) and needed > 0
