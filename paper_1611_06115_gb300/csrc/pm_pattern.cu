// Pattern coding (Sec. 2.2, Table 2) into per-chunk membership masks.
//
// Sec. 2 keeps, of the prime coding of Sec. 1.3, only whether each (pattern
// symbol, text letter) pair leaves residue 0 modulo M.  This file derives
// that bit the same way: with one prime per letter (2, 3, 5, 7 for A, C, G,
// T; any four distinct primes will do for single pairs), a class S gets the
// code n_S of Eq. 1 by the Chinese remainder theorem, letter a the code
// e_a = M / k_a of Sec. 1.3.1, and a belongs to S iff e_a * n_S = 0 (mod M)
// (Eq. 3 for a single pair).  The resulting 4-bit masks are the rows of
// Table 3 with 0 and 1 swapped.  The class letters are the "Character class"
// column of Table 2; any other byte has the empty class, i.e. the code 1111
// ("-") that Sec. 2.2 gives to missing or erroneous symbols.
#include <cstring>
#include <new>

#include "pm_internal.cuh"

namespace pm {
namespace {

struct ClassRow {
    char symbol;
    const char *letters;
};

// Table 2, "Character class" and "Symbol" columns.
constexpr ClassRow kTable2[] = {
    {'A', "A"},   {'C', "C"},   {'G', "G"},   {'T', "T"},   {'M', "AC"},  {'R', "AG"},
    {'W', "AT"},  {'S', "CG"},  {'Y', "CT"},  {'K', "GT"},  {'V', "ACG"}, {'H', "ACT"},
    {'D', "AGT"}, {'B', "CGT"}, {'N', "ACGT"}, {'-', ""},
};

constexpr uint64_t kPrime[4] = {2, 3, 5, 7};  // letters A, C, G, T (Table 1 order)

uint64_t inverse_mod(uint64_t a, uint64_t q)
{
    for (uint64_t x = 1; x < q; ++x)
        if ((a * x) % q == 1) return x;
    return 0;
}

// Eq. 1 by the CRT, then the residue test of Eq. 3 for each letter.
uint8_t residue_membership(const char *letters)
{
    uint64_t M = 1;
    for (uint64_t q : kPrime) M *= q;
    uint64_t nS = 0;
    for (int i = 0; i < 4; ++i) {
        const bool in = std::strchr(letters, "ACGT"[i]) != nullptr;
        const uint64_t Mi = M / kPrime[i];
        nS += (in ? 0 : 1) * Mi * inverse_mod(Mi % kPrime[i], kPrime[i]);
    }
    nS %= M;
    uint8_t mask = 0;
    for (int a = 0; a < 4; ++a) {
        const uint64_t e = M / kPrime[a];
        if ((e * nS) % M == 0) mask |= (uint8_t)(1u << a);
    }
    return mask;
}

struct MembershipTable {
    uint8_t mask[256];
    bool known[256];
    MembershipTable()
    {
        std::memset(mask, 0, sizeof mask);
        std::memset(known, 0, sizeof known);
        for (const ClassRow &r : kTable2) {
            const uint8_t m = residue_membership(r.letters);
            const unsigned char up = (unsigned char)r.symbol;
            mask[up] = m;
            known[up] = true;
            if (up >= 'A' && up <= 'Z') {
                mask[up - 'A' + 'a'] = m;
                known[up - 'A' + 'a'] = true;
            }
        }
    }
};

const MembershipTable &membership()
{
    static const MembershipTable t;
    return t;
}

}  // namespace
}  // namespace pm

using namespace pm;

extern "C" {

pm_status pm_compile_pattern(const char *iupac, uint32_t m, pm_pattern **out)
{
    if (!out || !iupac || m == 0) {
        set_error("pm_compile_pattern: NULL argument or m == 0");
        return PM_E_ARG;
    }
    *out = nullptr;
    if (m > PM_MAX_PATTERN) {
        set_error("pm_compile_pattern: m = %u exceeds %u", m, PM_MAX_PATTERN);
        return PM_E_TOO_LARGE;
    }
    const MembershipTable &tab = membership();
    pm_pattern *p = new (std::nothrow) pm_pattern{};
    if (!p) return PM_E_NOMEM;
    p->m = m;
    p->nchunks = (m + 31) / 32;
    p->masks = new (std::nothrow) uint4[p->nchunks];
    if (!p->masks) {
        delete p;
        return PM_E_NOMEM;
    }
    for (uint32_t c = 0; c < p->nchunks; ++c) p->masks[c] = make_uint4(0, 0, 0, 0);
    for (uint32_t j = 0; j < m; ++j) {
        const unsigned char ch = (unsigned char)iupac[j];
        if (!tab.known[ch]) ++p->unknown;
        const uint8_t mask = tab.mask[ch];
        const uint32_t bit = 1u << (j & 31);
        uint4 &w = p->masks[j >> 5];
        if (mask & 1) w.x |= bit;
        if (mask & 2) w.y |= bit;
        if (mask & 4) w.z |= bit;
        if (mask & 8) w.w |= bit;
    }
    // positions past m match every letter
    for (uint32_t j = m; j < 32 * p->nchunks; ++j) {
        const uint32_t bit = 1u << (j & 31);
        uint4 &w = p->masks[j >> 5];
        w.x |= bit; w.y |= bit; w.z |= bit; w.w |= bit;
    }
    // window-sliced position list (first 32 positions)
    const uint32_t head = m < 32 ? m : 32;
    p->wslist = new (std::nothrow) uint4[2 * head + 1];
    if (!p->wslist) {
        delete[] p->masks;
        delete p;
        return PM_E_NOMEM;
    }
    // one-letter classes first (the most selective), each as its letter's
    // Table 1 code (the end of its run is set when the list is ordered)
    for (uint32_t j = 0; j < head; ++j) {
        const uint8_t mask = tab.mask[(unsigned char)iupac[j]];
        if (__builtin_popcount(mask) != 1) continue;
        const uint32_t code = (uint32_t)__builtin_ctz(mask);  // A=0 C=1 G=2 T=3
        p->wslist[p->n_single++] = make_uint4(j, code, 0u, 0u);
    }
    // then the other classes except N (which never mismatches), as membership words
    for (uint32_t j = 0; j < head; ++j) {
        const uint8_t mask = tab.mask[(unsigned char)iupac[j]];
        if (mask == 0xf || __builtin_popcount(mask) == 1) continue;
        uint4 *e = p->wslist + p->n_single + 2 * p->n_general++;
        e[0] = make_uint4(j, 0u, 0u, 0u);
        e[1] = make_uint4(0u - (mask & 1u), 0u - ((mask >> 1) & 1u), 0u - ((mask >> 2) & 1u),
                          0u - ((mask >> 3) & 1u));
    }
    *out = p;
    return PM_OK;
}

uint32_t pm_pattern_length(const pm_pattern *p) { return p ? p->m : 0; }
uint32_t pm_pattern_unknown(const pm_pattern *p) { return p ? p->unknown : 0; }

pm_status pm_pattern_masks(const pm_pattern *p, uint32_t *out, uint64_t words)
{
    if (!p || !out || words < 4ull * p->nchunks) {
        set_error("pm_pattern_masks: NULL argument or too few words");
        return PM_E_ARG;
    }
    std::memcpy(out, p->masks, sizeof(uint4) * p->nchunks);
    return PM_OK;
}

void pm_pattern_free(pm_pattern *p)
{
    if (!p) return;
    delete[] p->masks;
    delete[] p->wslist;
    delete p;
}

}  // extern "C"
