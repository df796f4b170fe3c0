"""Failure detection without a GPU fault: the bounded barrier wait that any
kernel waiting on a bulk copy's barrier uses gives up after its limit when
nothing completes the barrier, the kernel returns, and the context stays
usable; capacity overflows and bad arguments come back as status codes."""
import time

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


def test_wait_that_nothing_completes_times_out_and_returns(pm):
    t0 = time.perf_counter()
    assert pm.api.pm_check_bounded_wait(2_000_000, arrive=False) is True  # 2 ms limit
    dt = time.perf_counter() - t0
    assert dt < 5.0
    assert pm.api.pm_check_bounded_wait(2_000_000, arrive=True) is False
    with pytest.raises(pm.PmError) as e:
        pm.api.pm_check_bounded_wait(0, arrive=False)
    assert e.value.status == pm.PM_E_ARG
    # the context is still usable: a search right after gives the oracle's hits
    text = synth.markov_text(4096 * 32 + 9, seed=3)
    t = pm.pm_encode_text(text)
    r = pm.pm_search(t, [pm.pm_compile_pattern("ACGTRYACGT")], [2])
    l, c = r.pattern(0)
    el, ec = oracle.search(text, "ACGTRYACGT", 2)
    assert np.array_equal(l, el) and np.array_equal(c, ec)


def test_status_codes_instead_of_faults(pm):
    import torch
    text = synth.markov_text(50_000, seed=4)
    t = pm.pm_encode_text(text)
    p = pm.pm_compile_pattern("ACGTNNAC")
    with pytest.raises(pm.PmError) as e:  # too small an output
        pm.pm_search_ex(t, [p], [3], capacity=1, out="host")
    assert e.value.status == pm.PM_E_OVERFLOW
    with pytest.raises(pm.PmError) as e:  # unknown variant
        pm.pm_search_ex(t, [p], [3], variant=9)
    assert e.value.status == pm.PM_E_ARG
    with pytest.raises(pm.PmError) as e:  # negative k
        pm.pm_search(t, [p], [-1])
    assert e.value.status == pm.PM_E_ARG
    with pytest.raises(pm.PmError) as e:  # batch option out of range
        pm.Batch(t, [p], [3], capacity=10, tiles=65)
    assert e.value.status == pm.PM_E_ARG
    with pytest.raises(pm.PmError) as e:  # a symbol outside Table 1
        pm.pm_encode_text(b"ACGTX")
    assert e.value.status == pm.PM_E_SYMBOL
    torch.cuda.synchronize()


@pytest.mark.parametrize("batch", (None, {}))
def test_outputs_are_written_within_their_bounds(pm, batch):
    """Canary records after the capacity and after offsets[npat] stay as
    they were: the kernels write nothing past what the call was given, also
    when the output does not fit."""
    import torch
    rng = np.random.default_rng(8)
    text = synth.markov_text(3 * 4096 * 32 + 5, seed=8)
    t = pm.pm_encode_text(text)
    pats = [synth.random_pattern(m, m // 10, rng) for m in (12, 40, 90)]
    ks = [2, 6, 14]
    cps = [pm.pm_compile_pattern(p) for p in pats]
    total = pm.pm_search(t, cps, ks).total
    for cap in (total, total + 10, max(total // 2, 1)):
        pad = 257
        hits = torch.full((cap + pad, 2), -7, dtype=torch.int32, device="cuda")
        offs = torch.full((len(cps) + 1 + pad,), -9, dtype=torch.int64, device="cuda")
        L = pm.lib()
        import ctypes
        harr = (ctypes.c_void_p * len(cps))(*[c.handle for c in cps])
        karr = (ctypes.c_int32 * len(ks))(*ks)
        bopts = pm._native.pm_batch_options() if batch is not None else None
        opts = pm._native.pm_options(0, 0, None, ctypes.pointer(bopts) if bopts is not None else None)
        needed = ctypes.c_uint64(0)
        st = L.pm_search_ex(t.handle, harr, len(cps), karr, ctypes.c_void_p(hits.data_ptr()), cap,
                            ctypes.c_void_p(offs.data_ptr()), ctypes.byref(needed), ctypes.byref(opts),
                            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        torch.cuda.synchronize()
        assert needed.value == total
        assert st == (0 if total <= cap else pm.PM_E_OVERFLOW)
        assert (hits[cap:] == -7).all()
        if total > cap:
            assert (hits[:cap] == -7).all()       # nothing written when the output does not fit
        else:
            assert (hits[total:cap] == -7).all()  # nothing past the hits found
        assert (offs[len(cps) + 1:] == -9).all()
