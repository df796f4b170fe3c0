/*
 * The C ABI used from plain C (no Python): the worked example of Sec. 2.5
 * (pattern C[CGT]GG[CG] over ATGACCGGCAT; 1-based hits 5 at k = 0 and
 * 1, 4, 5, 6 at k = 2), host outputs, an overflow that reports the count it
 * needs, and a text with an unknown symbol.  Exit status 0 when every check
 * holds; a message on stderr otherwise.
 */
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include "pm.h"

#define CHECK(cond, ...)                                      \
    do {                                                      \
        if (!(cond)) {                                        \
            fprintf(stderr, "abi_example: " __VA_ARGS__);     \
            fprintf(stderr, " (%s)\n", pm_last_error());      \
            return 1;                                         \
        }                                                     \
    } while (0)

int main(void)
{
    const char *t = "ATGACCGGCAT";
    const char *p = "CBGGS";  /* C [CGT] G G [CG] */
    pm_text *text = NULL;
    pm_pattern *pat = NULL;
    CHECK(pm_encode_text(t, strlen(t), NULL, &text) == PM_OK, "pm_encode_text failed");
    CHECK(pm_compile_pattern(p, (uint32_t)strlen(p), &pat) == PM_OK, "pm_compile_pattern failed");

    const pm_pattern *pats[2] = {pat, pat};
    const int32_t k[2] = {0, 2};
    pm_hit hits[16];
    uint64_t offsets[3], needed = 0;
    CHECK(pm_search(text, pats, 2, k, hits, 16, offsets, &needed, NULL) == PM_OK, "pm_search failed");
    CHECK(needed == 5 && offsets[0] == 0 && offsets[1] == 1 && offsets[2] == 5,
          "offsets %llu %llu %llu, needed %llu", (unsigned long long)offsets[0],
          (unsigned long long)offsets[1], (unsigned long long)offsets[2], (unsigned long long)needed);
    CHECK(hits[0].location + 1 == 5 && hits[0].mismatches == 0, "k = 0 hit");
    const uint32_t want[4] = {1, 4, 5, 6};
    for (int i = 0; i < 4; ++i)
        CHECK(hits[1 + i].location + 1 == want[i], "k = 2 hit %d at %u", i, hits[1 + i].location + 1);

    /* too small a capacity: nothing written, the count needed reported */
    CHECK(pm_search(text, pats, 2, k, hits, 3, offsets, &needed, NULL) == PM_E_OVERFLOW && needed == 5,
          "overflow not reported");

    /* a symbol outside Table 1: an error by default, unknown on request */
    pm_text *bad = NULL;
    CHECK(pm_encode_text("ACGNT", 5, NULL, &bad) == PM_E_SYMBOL, "N accepted by pm_encode_text");
    CHECK(pm_encode_text_ex("ACGNT", 5, PM_TEXT_UNKNOWN_AS_N, NULL, &bad) == PM_OK && pm_text_unknown(bad) == 1,
          "pm_encode_text_ex");
    pm_pattern *nn = NULL, *gg = NULL;
    CHECK(pm_compile_pattern("GN", 2, &nn) == PM_OK && pm_compile_pattern("GA", 2, &gg) == PM_OK, "compile");
    const pm_pattern *two[2] = {nn, gg};
    const int32_t k0[2] = {0, 0};
    CHECK(pm_search(bad, two, 2, k0, hits, 16, offsets, &needed, NULL) == PM_OK, "search unknown");
    /* "GN" matches G followed by the unknown symbol; "GA" does not */
    CHECK(offsets[1] == 1 && hits[0].location == 2 && offsets[2] == 1, "unknown-symbol hits");

    pm_pattern_free(nn);
    pm_pattern_free(gg);
    pm_text_free(bad);
    pm_pattern_free(pat);
    pm_text_free(text);
    puts("abi_example ok");
    return 0;
}
