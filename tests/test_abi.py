"""The C ABI without a GPU: the library builds, loads, exports every function
include/pm.h declares, and its host-only pattern compiler (Sec. 2.2) gives
the membership of Table 3 as the oracle holds it."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
from oracle import linhart_shamir as ls

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SYMBOLS = "ACGTMRWSYKVHDBN-"


def declared_functions():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b(pm_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def libpm():
    from paper_1611_06115_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for need in ("pm_encode_text", "pm_compile_pattern", "pm_search", "pm_text_free",
                 "pm_pattern_free", "pm_status_string"):
        assert need in names


def test_library_exports_every_declared_function(libpm):
    missing = [n for n in sorted(declared_functions()) if not hasattr(libpm, n)]
    assert not missing, missing


def test_binding_covers_every_declared_function():
    from paper_1611_06115_gb300 import _native
    assert declared_functions() <= set(_native.SIGNATURES)


def test_status_strings(libpm):
    import paper_1611_06115_gb300 as pm
    L = pm.lib()
    for s in range(0, -8, -1):
        assert L.pm_status_string(s).decode() not in ("", "unknown status")
    assert L.pm_status_string(-99).decode() == "unknown status"


def test_compiled_masks_equal_table3():
    """Each compiled class mask is the complement of the oracle's Table 3 row."""
    import paper_1611_06115_gb300 as pm
    L = oracle.table3()
    pat = (SYMBOLS * 3)[:40] + "xz"
    p = pm.pm_compile_pattern(pat)
    assert p.m == len(pat) and p.unknown == 2
    M = p.masks()
    for j, ch in enumerate(pat):
        for a, letter in enumerate("ACGT"):
            bit = (int(M[j // 32, a]) >> (j % 32)) & 1
            l = oracle.lindex(oracle.pattern_code(ch), oracle.text_code(letter))
            assert bit == 1 - L[l], (j, ch, letter)
    # positions past m match everything
    for j in range(len(pat), 32 * M.shape[0]):
        assert all((int(M[j // 32, a]) >> (j % 32)) & 1 for a in range(4))


def test_compiled_masks_lowercase_and_prime_test():
    import paper_1611_06115_gb300 as pm
    up = pm.pm_compile_pattern("ACGTMRWSYKVHDBN-").masks()
    low = pm.pm_compile_pattern("acgtmrwsykvhdbn-").masks()
    assert np.array_equal(up, low)
    primes = ls.smallest_primes_above(16)
    for j, X in enumerate("ACGTMRWSYKVHDBN-"):
        for a, letter in enumerate("ACGT"):
            assert ((int(up[0, a]) >> j) & 1) == ls.pair_is_match(letter, X, primes)


def test_compile_argument_errors():
    import paper_1611_06115_gb300 as pm
    with pytest.raises(pm.PmError) as e:
        pm.pm_compile_pattern("")
    assert e.value.status == pm.PM_E_ARG
