"""GB300-native k-mismatch matching of IUPAC character-class patterns against a
2-bit DNA text, after "Fast low-level pattern matching algorithm" (Soldo,
Krzic, Sersic; arXiv 1611.06115).

Location i of a text holds a pattern with at most k mismatches when
``sum_j L[(p[j] << 2) OR t[i+j-1]] <= k`` (Eq. 4), with the text coded by
Table 1, the pattern by Table 2 and L the Table 3 dictionary, i.e. the
prime-residue class test of Sec. 1.3.  All of it runs in hand-written sm_103a
CUDA kernels behind the C ABI of ``include/pm.h`` (``libpm.so``); this package
is the Python binding, with the same names.
"""
from ._native import (PM_E_ARG, PM_E_CUDA, PM_E_NOMEM, PM_E_OVERFLOW, PM_E_SYMBOL,  # noqa: F401
                      PM_E_TIMEOUT, PM_E_TOO_LARGE, PM_OK, PM_TOTAL_ERROR,
                      PM_TEXT_UNKNOWN_AS_N, PM_VARIANT_ALL_CHUNKS, PM_VARIANT_AUTO,
                      PM_VARIANT_PATTERN_SLICED,
                      PM_VARIANT_PATTERN_SLICED_2, PM_VARIANT_WINDOW_SLICED,
                      NativeLibraryMissing, PmError, lib)
from .api import (Batch, GraphedBatch, Pattern, SearchResult, Text,  # noqa: F401
                  pm_compile_pattern, pm_encode_text, pm_encode_text_ex, pm_get_auto_variants,
                  pm_search,
                  pm_search_ex, pm_set_auto_variants)
