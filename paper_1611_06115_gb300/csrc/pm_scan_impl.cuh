// Device building blocks shared by the per-pattern and the batched scan
// kernels (see pm_scan.cu for the method they implement).
#pragma once

#include "pm_internal.cuh"

namespace pm {
namespace scan {

using dev::class_match;

constexpr uint32_t kFull = 0xffffffffu;
constexpr int G = kGroups;  // groups per warp tile of the batched kernel; the per-pattern
                            // kernels take theirs as a template parameter

// Mismatch count of window 32*blk + w over chunks c0.., starting from
// `count`, stopping once it exceeds `limit` (then some value > limit).
__device__ __forceinline__ uint32_t window_count_from(const uint2 *__restrict__ planes,
                                                      uint64_t blk, uint32_t w,
                                                      const uint4 *__restrict__ M,
                                                      uint32_t c0, uint32_t nchunks,
                                                      uint32_t count, uint32_t limit)
{
    uint2 a = __ldg(planes + blk + c0);
    for (uint32_t c = c0; c < nchunks; ++c) {
        const uint2 b = __ldg(planes + blk + c + 1);
        const uint32_t lo = __funnelshift_r(a.x, b.x, w);
        const uint32_t hi = __funnelshift_r(a.y, b.y, w);
        count += __popc(~class_match(lo, hi, __ldg(M + c)));
        if (count > limit) break;
        a = b;
    }
    return count;
}

// The exact count of window 32*blk + w (stopping once past `limit`) for a
// text that may hold unknown symbols (unk: one bit per symbol, NULL when the
// text has none).  At an unknown symbol only the class N (every letter)
// matches.  The planes code an unknown symbol as some letter, so the count
// the scan evaluations see there is never above this one: a window they
// drop is past k here too, and the windows they pass are recounted here.
__device__ __forceinline__ uint32_t window_count_exact(const uint2 *__restrict__ planes,
                                                       const uint32_t *__restrict__ unk,
                                                       uint64_t blk, uint32_t w,
                                                       const uint4 *__restrict__ M,
                                                       uint32_t nchunks, uint32_t limit)
{
    if (!unk) return window_count_from(planes, blk, w, M, 0, nchunks, 0u, limit);
    uint32_t count = 0;
    uint2 a = __ldg(planes + blk);
    uint32_t ua = __ldg(unk + blk);
    for (uint32_t c = 0; c < nchunks; ++c) {
        const uint2 b = __ldg(planes + blk + c + 1);
        const uint32_t ub = __ldg(unk + blk + c + 1);
        const uint4 Mc = __ldg(M + c);
        const uint32_t match = class_match(__funnelshift_r(a.x, b.x, w), __funnelshift_r(a.y, b.y, w), Mc);
        const uint32_t u = __funnelshift_r(ua, ub, w);
        const uint32_t is_n = Mc.x & Mc.y & Mc.z & Mc.w;  // also every position past m
        count += __popc(~((match & ~u) | (u & is_n)));
        if (count > limit) break;
        a = b;
        ua = ub;
    }
    return count;
}

// Drop from pass the windows whose exact count (window_count_exact) is past
// k; only texts with unknown symbols need it.
__device__ __forceinline__ uint32_t recount_unknown(uint32_t pass, const uint2 *__restrict__ planes,
                                                   const uint32_t *__restrict__ unk, uint64_t blk,
                                                   const uint4 *__restrict__ M, uint32_t nchunks,
                                                   uint32_t k)
{
    uint32_t sv = pass;
    while (sv) {
        const uint32_t w = __ffs(sv) - 1;
        sv &= sv - 1;
        if (window_count_exact(planes, unk, blk, w, M, nchunks, k) > k) pass &= ~(1u << w);
    }
    return pass;
}

__device__ __forceinline__ uint32_t mad_lo(uint32_t a, uint32_t b, uint32_t c)
{
    uint32_t r;
    asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(c));
    return r;
}

// Pattern-sliced test of the first C chunks (C = 1 or 2) for one lane's 32
// windows; pass mask (window w at bit w) of the windows with at most k
// mismatches in positions 0..32C-1 (k <= 32C-1).  Blocks blk, blk+1 (and
// blk+2 for C = 2) are a, b, c; M0, M1 the masks of chunks 0 and 1.  Step j
// takes windows j, 8 + j, 16 + j, 24 + j, one per byte of a multiply-add
// result that holds matches + k, below 2^(5+C) so bytes never carry: its
// bit 4+C is set exactly when matches + k >= 32C, i.e. when the window has
// at most k mismatches, and moves to bit 8q + j, the window's own bit.
// k4 = k in every byte; one, m8, m16, m24 = 1, 2^8, 2^16, 2^24.
template <int C>
__device__ __forceinline__ uint32_t pass_pattern_sliced(uint2 a, uint2 b, uint2 c, uint4 M0,
                                                        uint4 M1, uint32_t k4, uint32_t one,
                                                        uint32_t m8, uint32_t m16, uint32_t m24)
{
    static_assert(C == 1 || C == 2, "one or two chunks");
    constexpr int kBit = 4 + C;
    uint32_t pass = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        uint32_t g[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int w = 8 * q + j;
            g[q] = __popc(class_match(__funnelshift_r(a.x, b.x, w), __funnelshift_r(a.y, b.y, w), M0));
            if constexpr (C == 2)
                g[q] += __popc(class_match(__funnelshift_r(b.x, c.x, w), __funnelshift_r(b.y, c.y, w), M1));
        }
        uint32_t v = mad_lo(g[3], m24, k4);
        v = mad_lo(g[2], m16, v);
        v = mad_lo(g[1], m8, v);
        v = mad_lo(g[0], one, v);
        // bit kBit of byte q: g[q] + k >= 32C; move bits 8q + kBit to 8q + j = w
        const uint32_t s = j <= kBit ? v >> (kBit - j) : v << (j - kBit);
        pass |= s & (0x01010101u << j);
    }
    return pass;
}

// A position-list entry (the compact words of ordered_wslist) from shared
// memory, or from global memory through the read-only path (every lane reads
// the same address: one broadcast).
template <bool kGlobal>
__device__ __forceinline__ uint32_t ld_list(const uint32_t *p)
{
    if constexpr (kGlobal) return __ldg(p);
    else return *p;
}

// List entries the window-sliced scan tests before it leaves the remaining
// candidates to exact one-by-one counts (checked every four entries).
// Measured on GB300 over a 3.1 Gbp text (m = 32 .. 1024): K = 0 8 entries
// (2-3 % faster than no cut), K = 1..4 4 + 2K (7, 18, 4, 12 % faster); a
// cut one block earlier leaves so many candidates that their serial counts
// cost 1.4-4x the scan.  From K = 4 on (binary counters, blocks of four
// entries) 4 + 2K rounded down to a whole block: K = 5 m = 1024 0.71 -> 0.65
// ms, the other K and m unchanged.
__host__ __device__ constexpr uint32_t ws_cut(int K)
{
    return K == 0 ? 8u : (K >= 4 ? (4u + 2u * (uint32_t)K) & ~3u : 4u + 2u * (uint32_t)K);
}

// From this K on the window-sliced scan counts in binary (alive_window_sliced_bin).
constexpr int kWsBinaryFrom = 4;

// Bit i set where symbol i of block t is the letter with Table 1 code CODE
// (A = 00, C = 01, G = 10, T = 11; t.x holds the low code bits, t.y the high).
template <int CODE>
__device__ __forceinline__ uint32_t letter_plane(uint2 t)
{
    static_assert(CODE >= 0 && CODE < 4, "Table 1 codes");
    if constexpr (CODE == 0) return ~(t.x | t.y);
    else if constexpr (CODE == 1) return t.x & ~t.y;
    else if constexpr (CODE == 2) return ~t.x & t.y;
    else return t.x & t.y;
}

// Thermometer counter of K+1 levels over 32 windows: level i is set once a
// window has more than i mismatches.  `match` has bit w set where window w
// matches the position just tested.
template <int K>
__device__ __forceinline__ void add_position(uint32_t (&L)[K + 1], uint32_t match)
{
#pragma unroll
    for (int i = K; i >= 1; --i) L[i] |= L[i - 1] & ~match;
    L[0] |= ~match;
}

// True when every window of the lane's groups, on every lane, is past K.
template <int K, int G>
__device__ __forceinline__ bool all_past(const uint32_t (&L)[G][K + 1])
{
    uint32_t d = kFull;
#pragma unroll
    for (int g = 0; g < G; ++g) d &= L[g][K];
    return __all_sync(kFull, d == kFull);
}

// Outcome of a stretch of the window-sliced scan.
constexpr int kWsGoOn = 0;  // list not exhausted, some window alive
constexpr int kWsDead = 1;  // every window past K
constexpr int kWsCut = 2;   // `cut` entries tested, some window alive

// One run of list entries that share the one-letter class CODE (entries
// e .. end-1).  The letter's plane is built once per run from the lane's
// two blocks per group, so each position costs one funnel shift (its match
// word for 32 windows) and the counter update; K = 0 folds two positions
// into one update.  The early stop is checked whenever e reaches a multiple
// of the block size S (2 entries for K = 0 from entry 4 on, else 4), across
// run boundaries, as if the list were one run.
template <int K, int CODE, bool kGlobal, int G>
__device__ __forceinline__ int ws_letter_run(const uint2 (&a)[G], const uint2 (&b)[G],
                                             const uint32_t *__restrict__ list, uint32_t &e,
                                             uint32_t end, uint32_t cut, uint32_t (&L)[G][K + 1])
{
    uint32_t pa[G], pb[G];
#pragma unroll
    for (int g = 0; g < G; ++g) {
        pa[g] = letter_plane<CODE>(a[g]);
        pb[g] = letter_plane<CODE>(b[g]);
    }
    constexpr uint32_t S = K == 0 ? 2u : 4u;
    // Only k = 0 checks whether every window died: for k >= 1 a tile of
    // 4096 windows practically never dies whole before the cut.
    auto check = [&]() -> int {
        if (K == 0 && e < 4) return kWsGoOn;
        if (K == 0 && all_past<K, G>(L)) return kWsDead;
        if (e >= cut) return kWsCut;
        return kWsGoOn;
    };
    // single entries up to the next multiple of S
    while (e < end && (e & (S - 1)) != 0) {
        const uint32_t s0 = ld_list<kGlobal>(list + e);  // bits 0-4 the shift (taken modulo 32)
#pragma unroll
        for (int g = 0; g < G; ++g) add_position<K>(L[g], __funnelshift_r(pa[g], pb[g], s0));
        ++e;
        if ((e & (S - 1)) == 0) {
            const int r = check();
            if (r != kWsGoOn) return r;
        }
    }
    // whole blocks
    while (e + S <= end) {
        uint32_t s[S];
#pragma unroll
        for (uint32_t u = 0; u < S; ++u) s[u] = ld_list<kGlobal>(list + e + u);
#pragma unroll
        for (int g = 0; g < G; ++g) {
            if constexpr (K == 0) {
                L[g][0] |= ~(__funnelshift_r(pa[g], pb[g], s[0]) & __funnelshift_r(pa[g], pb[g], s[1]));
            } else {
#pragma unroll
                for (uint32_t u = 0; u < S; ++u) add_position<K>(L[g], __funnelshift_r(pa[g], pb[g], s[u]));
            }
        }
        e += S;
        const int r = check();
        if (r != kWsGoOn) return r;
    }
    // the rest of the run (fewer than S entries: no multiple of S is reached)
    for (; e < end; ++e) {
        const uint32_t s0 = ld_list<kGlobal>(list + e);
#pragma unroll
        for (int g = 0; g < G; ++g) add_position<K>(L[g], __funnelshift_r(pa[g], pb[g], s0));
    }
    return kWsGoOn;
}

// Binary counters for the window-sliced scan with larger k: per group five
// bit planes c[0..4] hold, for each of 32 windows, its mismatches so far in
// binary (c[4] sticky: 16 or more).  Four positions are added at once by
// carry-save adders (eleven three-input logic operations), so a position
// costs about 2.75 of them whatever k is, against k+1 for the thermometer.
// m0..m3 are match words (bit set: the window matches that position); a
// padding position is all ones.
constexpr int kCtr = 5;
__device__ __forceinline__ void add_four(uint32_t (&c)[kCtr], uint32_t m0, uint32_t m1, uint32_t m2, uint32_t m3)
{
    const uint32_t x0 = ~m0, x1 = ~m1, x2 = ~m2, x3 = ~m3;    // mismatch words
    const uint32_t s1 = x0 ^ x1 ^ x2;                          // weight 1
    const uint32_t k1 = (x0 & x1) | (x0 & x2) | (x1 & x2);     // weight 2
    const uint32_t k2 = (c[0] & s1) | (c[0] & x3) | (s1 & x3); // weight 2
    c[0] = c[0] ^ s1 ^ x3;
    const uint32_t k3 = (c[1] & k1) | (c[1] & k2) | (k1 & k2); // weight 4
    c[1] = c[1] ^ k1 ^ k2;
    const uint32_t k4 = c[2] & k3;                             // weight 8
    c[2] ^= k3;
    const uint32_t k5 = c[3] & k4;                             // weight 16
    c[3] ^= k4;
    c[4] |= k5;
}

// Windows whose count in c is above the compile-time K (K < 16).
template <int K>
__device__ __forceinline__ uint32_t count_above(const uint32_t (&c)[kCtr])
{
    static_assert(K >= 0 && K < 16, "four counter bits plus the sticky one");
    uint32_t gt = 0u, eq = kFull;
#pragma unroll
    for (int i = 3; i >= 0; --i) {
        if ((K >> i) & 1) {
            eq &= c[i];
        } else {
            gt |= eq & c[i];
            eq &= ~c[i];
        }
    }
    return gt | c[4];
}

// One run of one-letter entries e .. end-1 (letter CODE) added to the binary
// counters four at a time (the last block of the run padded with matching
// positions), until `cut` entries are done.
template <int CODE, bool kGlobal, int G>
__device__ __forceinline__ int ws_letter_run_bin(const uint2 (&a)[G], const uint2 (&b)[G],
                                                 const uint32_t *__restrict__ list, uint32_t &e,
                                                 uint32_t end, uint32_t cut, uint32_t (&C)[G][kCtr])
{
    uint32_t pa[G], pb[G];
#pragma unroll
    for (int g = 0; g < G; ++g) {
        pa[g] = letter_plane<CODE>(a[g]);
        pb[g] = letter_plane<CODE>(b[g]);
    }
    // whole blocks of four, then the run's last block padded with matches
    while (e + 4 <= end) {
        uint32_t s[4];
#pragma unroll
        for (uint32_t u = 0; u < 4; ++u) s[u] = ld_list<kGlobal>(list + e + u);
#pragma unroll
        for (int g = 0; g < G; ++g)
            add_four(C[g], __funnelshift_r(pa[g], pb[g], s[0]), __funnelshift_r(pa[g], pb[g], s[1]),
                     __funnelshift_r(pa[g], pb[g], s[2]), __funnelshift_r(pa[g], pb[g], s[3]));
        e += 4;
        if (e >= cut) return kWsCut;  // (no whole-tile early stop: see ws_letter_run)
    }
    if (e < end) {
        const uint32_t left = end - e;  // 1..3
        const uint32_t s0 = ld_list<kGlobal>(list + e);
        const uint32_t s1 = left > 1 ? ld_list<kGlobal>(list + e + 1) : 0u;
        const uint32_t s2 = left > 2 ? ld_list<kGlobal>(list + e + 2) : 0u;
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const uint32_t m1 = __funnelshift_r(pa[g], pb[g], s1), m2 = __funnelshift_r(pa[g], pb[g], s2);
            add_four(C[g], __funnelshift_r(pa[g], pb[g], s0), left > 1 ? m1 : kFull, left > 2 ? m2 : kFull, kFull);
        }
        e = end;
        if (e >= cut) return kWsCut;
    }
    return kWsGoOn;
}

// The window-sliced first chunk with binary counters, for 4 <= K < 16 (as
// alive_window_sliced, below, with the thermometer): the listed positions
// are added four at a time until ws_cut(K) entries are done or the list
// ends; alive[g] receives the windows still at or below K.  Returns true
// when it stopped at the cut with some window still alive.
template <int K, bool kGlobal, int G>
__device__ __forceinline__ bool alive_window_sliced_bin(const uint2 (&a)[G], const uint2 (&b)[G],
                                                        const uint32_t *__restrict__ list, uint32_t n_single,
                                                        uint32_t n_general, uint32_t cut,
                                                        const uint32_t (&valid)[G], uint32_t (&alive)[G])
{
    uint32_t C[G][kCtr];
#pragma unroll
    for (int g = 0; g < G; ++g) {
#pragma unroll
        for (int i = 0; i < kCtr - 1; ++i) C[g][i] = 0u;
        C[g][kCtr - 1] = ~valid[g];  // invalid windows count as past every K
    }
    uint32_t e = 0;
    bool stopped = false;
    while (e < n_single) {
        const uint32_t h = ld_list<kGlobal>(list + e);
        const uint32_t he = (h >> 8) & 63u;
        const uint32_t end = he > e ? (he < n_single ? he : n_single) : e + 1;
        int r;
        switch ((h >> 5) & 3u) {
        case 0: r = ws_letter_run_bin<0, kGlobal, G>(a, b, list, e, end, cut, C); break;
        case 1: r = ws_letter_run_bin<1, kGlobal, G>(a, b, list, e, end, cut, C); break;
        case 2: r = ws_letter_run_bin<2, kGlobal, G>(a, b, list, e, end, cut, C); break;
        default: r = ws_letter_run_bin<3, kGlobal, G>(a, b, list, e, end, cut, C); break;
        }
        if (r != kWsGoOn) {
            stopped = true;
            break;
        }
    }
    for (uint32_t c = 0; !stopped && c < n_general; c += 4) {
        const uint32_t left = n_general - c;
        uint32_t s[4];
#pragma unroll
        for (uint32_t u = 0; u < 4; ++u) s[u] = u < left ? ld_list<kGlobal>(list + n_single + c + u) : 0u;
#pragma unroll
        for (int g = 0; g < G; ++g) {
            uint32_t m[4];
#pragma unroll
            for (uint32_t u = 0; u < 4; ++u) {
                const uint4 M = make_uint4(0u - ((s[u] >> 16) & 1u), 0u - ((s[u] >> 17) & 1u),
                                           0u - ((s[u] >> 18) & 1u), 0u - ((s[u] >> 19) & 1u));
                m[u] = u < left ? class_match(__funnelshift_r(a[g].x, b[g].x, s[u]),
                                              __funnelshift_r(a[g].y, b[g].y, s[u]), M)
                                : kFull;
            }
            add_four(C[g], m[0], m[1], m[2], m[3]);
        }
        if (n_single + c + 4 >= cut && c + 4 < n_general) stopped = true;
    }
#pragma unroll
    for (int g = 0; g < G; ++g) alive[g] = ~count_above<K>(C[g]);
    // (stopped at the cut just as the list ended: alive is exact, and the
    // caller's settling of it is merely redundant)
    return stopped;
}

// Window-sliced first chunk with a thermometer counter of K+1 levels over the
// listed positions, for all groups of the lane at once.  The list (built by
// pm_compile_pattern, ordered for the text and packed by ordered_wslist)
// holds first the one-letter positions (shift, letter code, end of the run
// of that letter), grouped into runs by letter, then the other classes
// (shift, membership).  alive[g] receives the
// windows still at or below K.  After `cut` list entries the scan stops if
// some window is still alive and returns true: the few candidates left are
// cheaper to count one by one than to carry the whole tile through the
// remaining positions.  Returns false when every listed position was tested
// (alive is then exact over the first 32 positions) or every window died.
template <int K, bool kGlobal, int G>
__device__ __forceinline__ bool alive_window_sliced_thermo(const uint2 (&a)[G], const uint2 (&b)[G],
                                                           const uint32_t *__restrict__ list,
                                                           uint32_t n_single, uint32_t n_general,
                                                           uint32_t cut, const uint32_t (&valid)[G],
                                                           uint32_t (&alive)[G])
{
    uint32_t L[G][K + 1];
#pragma unroll
    for (int g = 0; g < G; ++g)
#pragma unroll
        for (int i = 0; i <= K; ++i) L[g][i] = ~valid[g];  // invalid windows sit at every level
    uint32_t e = 0;
    while (e < n_single) {
        const uint32_t h = ld_list<kGlobal>(list + e);
        // a run ends past its first entry and inside the list (also for a
        // malformed list, so that the loop always advances)
        const uint32_t he = (h >> 8) & 63u;
        const uint32_t end = he > e ? (he < n_single ? he : n_single) : e + 1;
        int r;
        switch ((h >> 5) & 3u) {
        case 0: r = ws_letter_run<K, 0, kGlobal, G>(a, b, list, e, end, cut, L); break;
        case 1: r = ws_letter_run<K, 1, kGlobal, G>(a, b, list, e, end, cut, L); break;
        case 2: r = ws_letter_run<K, 2, kGlobal, G>(a, b, list, e, end, cut, L); break;
        default: r = ws_letter_run<K, 3, kGlobal, G>(a, b, list, e, end, cut, L); break;
        }
        if (r != kWsGoOn) {
#pragma unroll
            for (int g = 0; g < G; ++g) alive[g] = r == kWsDead ? 0u : ~L[g][K];
            return r == kWsCut;
        }
    }
    for (uint32_t c = 0; c < n_general; ++c) {
        const uint32_t s = ld_list<kGlobal>(list + n_single + c);  // shift modulo 32
        const uint4 M = make_uint4(0u - ((s >> 16) & 1u), 0u - ((s >> 17) & 1u), 0u - ((s >> 18) & 1u),
                                   0u - ((s >> 19) & 1u));
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const uint32_t lo = __funnelshift_r(a[g].x, b[g].x, s);
            const uint32_t hi = __funnelshift_r(a[g].y, b[g].y, s);
            add_position<K>(L[g], class_match(lo, hi, M));
        }
        if ((c & 3) == 3) {
            if (K == 0 && all_past<K, G>(L)) {
#pragma unroll
                for (int g = 0; g < G; ++g) alive[g] = 0u;
                return false;
            }
            if (n_single + c + 1 >= cut) {
#pragma unroll
                for (int g = 0; g < G; ++g) alive[g] = ~L[g][K];
                return true;
            }
        }
    }
#pragma unroll
    for (int g = 0; g < G; ++g) alive[g] = ~L[g][K];
    return false;
}

// The window-sliced first chunk: a thermometer counter for K below
// kWsBinaryFrom (alive_window_sliced_thermo), binary counters from there on
// (alive_window_sliced_bin).
template <int K, bool kGlobal = false, int G>
__device__ __forceinline__ bool alive_window_sliced(const uint2 (&a)[G], const uint2 (&b)[G],
                                                    const uint32_t *__restrict__ list,
                                                    uint32_t n_single, uint32_t n_general,
                                                    uint32_t cut, const uint32_t (&valid)[G],
                                                    uint32_t (&alive)[G])
{
    if constexpr (K >= kWsBinaryFrom)
        return alive_window_sliced_bin<K, kGlobal, G>(a, b, list, n_single, n_general, cut, valid, alive);
    else
        return alive_window_sliced_thermo<K, kGlobal, G>(a, b, list, n_single, n_general, cut, valid, alive);
}

// Blocks a per-pattern scan stage holds: a warp tile of 32G blocks from an
// even block (the one at or below the tile's first block plus the first-stage
// chunk), the 2-block halo, and one more block so that the count is even.
template <int G>
__host__ __device__ constexpr uint32_t scan_stage_blocks() { return 32u * G + 4u; }

// One stage for the per-pattern scan, global -> shared, by the warp's own
// lanes: scan_stage_blocks<G>() blocks from block `first` (even, so that both
// addresses are 16-byte aligned) as 16-byte asynchronous copies (cp.async),
// lane l taking pieces l, l + 32, ... and lanes 0 and 1 the last two, as one
// commit group per lane.  Complete once every lane has passed cp_async_wait
// for the group and the warp has synchronised.
template <int G>
__device__ __forceinline__ void copy_tile_async(const uint2 *planes, uint64_t first, uint2 *dst, int lane)
{
    constexpr uint32_t kPieces = scan_stage_blocks<G>() / 2;  // 16 bytes each
    static_assert(kPieces == 16 * G + 2, "32 lanes take 16G pieces, lanes 0 and 1 the last two");
    const char *src = (const char *)(planes + first);
    const uint32_t d = dev::smem_u32(dst);
#pragma unroll
    for (uint32_t i = 0; i < 16u * G; i += 32u)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d + 16u * (i + lane)),
                     "l"(src + 16 * (i + lane))
                     : "memory");
    if (lane < 2)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d + 16u * (16u * G + lane)),
                     "l"(src + 16 * (16 * G + lane))
                     : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

// Wait until at most N of this lane's most recent commit groups are pending.
template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}


// Window-valid mask of the 32 windows that start in block blk.
__device__ __forceinline__ uint32_t valid_mask(uint64_t blk, uint64_t nwin)
{
    const uint64_t w0 = blk * 32ull;
    return w0 >= nwin ? 0u : (nwin - w0 >= 32 ? kFull : (1u << (uint32_t)(nwin - w0)) - 1u);
}

// Pattern-sliced evaluation over all chunks for large k (k > 31, where one
// chunk cannot decide a window): 32 per-window counts in registers, one
// chunk after another (chunk c needs blocks blk+c and blk+c+1; blocks 0 and
// 1 are given), until every window of the warp has passed k (the early stop
// of Sec. 2.4) or the pattern ends.  Returns the windows whose full count
// is at most k.
__device__ __forceinline__ uint32_t pass_multi_chunk(const uint2 *__restrict__ planes, uint64_t blk,
                                                     const uint4 *__restrict__ M, uint32_t nchunks,
                                                     uint32_t k, uint32_t valid, uint2 t0, uint2 t1)
{
    // counts only grow, so a window is a hit iff its final count is at most
    // k; the loop only needs the lane's smallest count to know whether any
    // of its windows is still at or below k (invalid windows start far past
    // any k, so they never keep it going)
    constexpr uint32_t kPast = 1u << 30;
    uint32_t cnt[32];
#pragma unroll
    for (int w = 0; w < 32; ++w) cnt[w] = (valid >> w) & 1u ? 0u : kPast;
    for (uint32_t c = 0; c < nchunks; ++c) {
        if (c > 0) {
            t0 = t1;
            t1 = __ldg(planes + blk + c + 1);
        }
        const uint4 Mc = __ldg(M + c);
        uint32_t low = kPast;
#pragma unroll
        for (int w = 0; w < 32; ++w) {
            cnt[w] += __popc(~class_match(__funnelshift_r(t0.x, t1.x, w), __funnelshift_r(t0.y, t1.y, w), Mc));
            low = min(low, cnt[w]);
        }
        if (!__any_sync(kFull, low <= k)) break;
    }
    uint32_t alive = 0;
#pragma unroll
    for (int w = 0; w < 32; ++w) alive |= (cnt[w] <= k ? 1u : 0u) << w;
    return alive;
}

// Exact counts of the windows still in `pass` for a pattern longer than 32:
// each lane counts its own remaining windows, chunk by chunk, and drops
// those past k.
__device__ __forceinline__ uint32_t settle_lane(uint32_t pass, uint64_t blk,
                                                const uint4 *__restrict__ M, uint32_t nchunks,
                                                uint32_t k, const uint2 *__restrict__ planes)
{
    uint32_t sv = pass;
    while (sv) {
        const uint32_t w = __ffs(sv) - 1;
        sv &= sv - 1;
        if (window_count_from(planes, blk, w, M, 0, nchunks, 0u, k) > k) pass &= ~(1u << w);
    }
    return pass;
}

// The count of window 32*blk + w, exact up to k (once past k, some value
// above k), when blocks blk+c0 and blk+c0+1 are at hand (t0, t1) and block
// blk+c0+2 is still staged at *s_t2: chunks c0 and c0+1 from those, the
// others through L1/L2 (rarely reached while k is below the expected
// mismatches of 64 positions).
__device__ __forceinline__ uint32_t count_from_first(uint2 t0, uint2 t1, const uint2 *s_t2, uint64_t blk,
                                                     uint32_t w, const uint4 *__restrict__ M, uint32_t c0,
                                                     uint32_t nchunks, uint32_t k,
                                                     const uint2 *__restrict__ planes)
{
    uint32_t c = __popc(~class_match(__funnelshift_r(t0.x, t1.x, w), __funnelshift_r(t0.y, t1.y, w), __ldg(M + c0)));
    if (c > k) return c;
    if (c0 + 1 < nchunks) {
        const uint2 t2 = *s_t2;
        c += __popc(~class_match(__funnelshift_r(t1.x, t2.x, w), __funnelshift_r(t1.y, t2.y, w),
                                 __ldg(M + c0 + 1)));
        if (c > k) return c;
    }
    if (c0 > 0) {
        c = window_count_from(planes, blk, w, M, 0, c0, c, k);
        if (c > k) return c;
    }
    if (c0 + 2 < nchunks) c = window_count_from(planes, blk, w, M, c0 + 2, nchunks, c, k);
    return c;
}

// Exact counts of the windows still in `pass` for a lane whose blocks
// blk+c0 and blk+c0+1 are in registers (t0, t1) and whose block blk+c0+2 is
// still staged in shared memory (s_next): drops those past k.
__device__ __forceinline__ uint32_t settle_staged(uint32_t pass, uint64_t blk, uint2 t0, uint2 t1,
                                                 const uint2 *s_next, const uint4 *__restrict__ M,
                                                 uint32_t c0, uint32_t nchunks, uint32_t k,
                                                 const uint2 *__restrict__ planes)
{
    uint32_t sv = pass;
    while (sv) {
        const uint32_t w = __ffs(sv) - 1;
        sv &= sv - 1;
        if (count_from_first(t0, t1, s_next, blk, w, M, c0, nchunks, k, planes) > k) pass &= ~(1u << w);
    }
    return pass;
}

// Exact counts of the windows still in `pass`, the first chunk from the
// lane's blocks in registers (t0, t1), the rest through L1/L2 (any m):
// drops those past k.
__device__ __forceinline__ uint32_t settle_from_regs(uint32_t pass, uint64_t blk, uint2 t0, uint2 t1,
                                                    const uint4 *__restrict__ M, uint32_t nchunks,
                                                    uint32_t k, const uint2 *__restrict__ planes)
{
    if (!pass) return 0u;
    const uint4 M0 = __ldg(M);
    uint32_t sv = pass;
    while (sv) {
        const uint32_t w = __ffs(sv) - 1;
        sv &= sv - 1;
        uint32_t c = __popc(~class_match(__funnelshift_r(t0.x, t1.x, w), __funnelshift_r(t0.y, t1.y, w), M0));
        if (c <= k && nchunks > 1) c = window_count_from(planes, blk, w, M, 1, nchunks, c, k);
        if (c > k) pass &= ~(1u << w);
    }
    return pass;
}

// Run-time constants of the pattern-sliced byte test for one k (k <= 63;
// the kernels use it only where k < 32C).
struct PsConst {
    uint32_t one, m8, m16, m24, k4;
};

__device__ __forceinline__ PsConst ps_const(uint32_t two, uint32_t k)
{
    PsConst c;
    c.one = two >> 1;
    c.m8 = c.one << 8;
    c.m16 = c.one << 16;
    c.m24 = c.one << 24;
    c.k4 = (k < 64u ? k : 0u) * (c.m24 | c.m16 | c.m8 | c.one);
    return c;
}

// First stage of one warp tile: pass[g] bit w for window 32*blk[g] + w,
// a superset of the windows of the tile that hold the pattern with at most k
// mismatches (VARIANT as in k_scan; list is the window-sliced position list
// in shared memory; stage the tile still staged in shared memory, from
// block tile*32G + d.c0 on; a[g], b[g] its blocks 32g + lane and 32g + lane
// + 1; M0 the masks of chunk d.c0, which the pattern-sliced evaluations test
// first, the others chunk 0).  Returns
// true when pass still needs exact counts past the positions tested (see
// settle_dense or settle_emit_queued); false when pass is exact.
template <int VARIANT, int G>
__device__ __forceinline__ bool tile_first_stage(const uint2 (&a)[G], const uint2 (&b)[G],
                                                 uint32_t tile, const uint32_t (&valid)[G],
                                                 const PatDesc &d, const uint4 *__restrict__ M,
                                                 uint4 M0, const uint32_t *__restrict__ list,
                                                 const PsConst &pc, const uint2 *__restrict__ planes,
                                                 const uint2 *stage, uint32_t (&pass)[G])
{
    const uint32_t k = (uint32_t)d.k;
    if constexpr (VARIANT >= 0) {
        const bool cut = alive_window_sliced<VARIANT>(a, b, list, d.n_single, d.n_general, ws_cut(VARIANT),
                                                      valid, pass);
        return cut || d.nchunks > 1;
    } else if constexpr (VARIANT == -2) {
        // k > 31: one chunk cannot decide; count all chunks (exact)
        const int lane = threadIdx.x & 31;
#pragma unroll 1
        for (int g = 0; g < G; ++g)
            pass[g] = pass_multi_chunk(planes, (uint64_t)tile * (32u * G) + 32u * g + lane, M, d.nchunks, k,
                                       valid[g], a[g], b[g]);
        return false;
    } else {
        // -1: one chunk; -3: two chunks (chunk 1 of a pattern with m <= 32
        // reads as all ones: every position past m matches)
        constexpr int C = VARIANT == -3 ? 2 : 1;
        const int lane = threadIdx.x & 31;
        const uint4 M1 = (C == 2 && d.c0 + 1 < d.nchunks) ? __ldg(M + d.c0 + 1)
                                                           : make_uint4(kFull, kFull, kFull, kFull);
#pragma unroll
        for (int g = 0; g < G; ++g) {
            uint32_t t = 0u;
            if (valid[g]) {
                const uint2 c = C == 2 ? stage[32 * g + lane + 2] : make_uint2(0u, 0u);
                t = pass_pattern_sliced<C>(a[g], b[g], c, M0, M1, pc.k4, pc.one, pc.m8, pc.m16,
                                           pc.m24) & valid[g];
            }
            pass[g] = t;
        }
        return d.nchunks > (uint32_t)C;  // (c0 > 0 only when nchunks > C)
    }
}

// Exact counts for pass (when `need`), each lane settling its own windows:
// the path for tiles with more candidates than settle_emit_queued takes.
template <int VARIANT, int G>
__device__ __forceinline__ void settle_dense(bool need, const uint2 (&a)[G], const uint2 (&b)[G],
                                             const uint64_t (&blk)[G], const PatDesc &d,
                                             const uint4 *__restrict__ M,
                                             const uint2 *__restrict__ planes, const uint2 *stage,
                                             uint32_t (&pass)[G])
{
    if (!need) return;
    const uint32_t k = (uint32_t)d.k;
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int g = 0; g < G; ++g) {
        if constexpr (VARIANT >= 0)
            pass[g] = settle_from_regs(pass[g], blk[g], a[g], b[g], M, d.nchunks, k, planes);
        else if constexpr (VARIANT == -1 || VARIANT == -3)
            pass[g] = settle_staged(pass[g], blk[g], a[g], b[g], stage + 32 * g + lane + 2, M, d.c0,
                                    d.nchunks, k, planes);
        else
            pass[g] = settle_lane(pass[g], blk[g], M, d.nchunks, k, planes);
    }
}

// Emit the hits of one warp tile in window order through one
// warp-aggregated atomic on cursor.  Call with the whole warp and only when
// some lane has a pass bit.  Returns (on every lane) the number of hits and
// where they start in tmp.
// kRegs: the lane's blocks a[g], b[g] (registers, blocks blk+c0 and
// blk+c0+1) and the still-staged tile (stage, from block tile*32G + d.c0 on)
// give chunks c0 and c0+1 of a hit's count without a load through L1/L2
// (other chunks, and texts with unknown symbols, count through L1/L2); hits
// are dense for small m and large k.  Otherwise every hit is counted through
// L1/L2, which keeps a and b out of registers during emission.
template <bool kRegs, int G>
__device__ __forceinline__ void emit_tile_hits(uint32_t (&pass)[G], const uint64_t (&blk)[G],
                                               const uint2 (&a)[G], const uint2 (&b)[G], const uint2 *stage,
                                               const PatDesc &d, const uint4 *__restrict__ M,
                                               const uint2 *__restrict__ planes,
                                               const uint32_t *__restrict__ unk,
                                               pm_hit *__restrict__ tmp, uint64_t cap,
                                               unsigned long long *__restrict__ cursor,
                                               uint32_t &total_out, unsigned long long &base_out)
{
    const int lane = threadIdx.x & 31;
    if (unk) {
#pragma unroll
        for (int g = 0; g < G; ++g)
            pass[g] = recount_unknown(pass[g], planes, unk, blk[g], M, d.nchunks, (uint32_t)d.k);
    }
    uint32_t incl[G], tot[G];
    uint32_t total = 0;
#pragma unroll
    for (int g = 0; g < G; ++g) {
        incl[g] = __popc(pass[g]);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t v = __shfl_up_sync(kFull, incl[g], o);
            if (lane >= o) incl[g] += v;
        }
        tot[g] = __shfl_sync(kFull, incl[g], 31);
        total += tot[g];
    }
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(cursor, (unsigned long long)total);
    base = __shfl_sync(kFull, base, 0);
    total_out = total;
    base_out = base;
#pragma unroll
    for (int g = 0; g < G; ++g) {
        unsigned long long q = base + incl[g] - __popc(pass[g]);
        uint32_t hm = pass[g];
        while (hm) {
            const uint32_t w = __ffs(hm) - 1;
            hm &= hm - 1;
            if (q < cap) {
                uint32_t c;
                if (!kRegs || unk) {
                    c = window_count_exact(planes, unk, blk[g], w, M, d.nchunks, (uint32_t)d.k);
                } else {
                    c = count_from_first(a[g], b[g], stage + 32 * g + lane + 2, blk[g], w, M, d.c0, d.nchunks,
                                         (uint32_t)d.k, planes);
                }
                tmp[q] = pm_hit{(uint32_t)(blk[g] * 32ull + w), c};
            }
            ++q;
        }
        base += tot[g];
    }
}

// Candidates a warp settles per tile through its shared-memory queue
// (settle_emit_queued); tiles with more take settle_dense and emit_tile_hits.
constexpr uint32_t kQueueCap = 256;

// The count of window 32*blk + w, exact up to k (once past k, some value
// above k), whose blocks blk+c0 .. blk+c0+2 are staged at stage_blk[0..2].
__device__ __forceinline__ uint32_t candidate_count(const uint2 *stage_blk, uint64_t blk, uint32_t w,
                                                    const uint4 *__restrict__ M, uint32_t c0,
                                                    uint32_t nchunks, uint32_t k,
                                                    const uint2 *__restrict__ planes,
                                                    const uint32_t *__restrict__ unk)
{
    if (unk) return window_count_exact(planes, unk, blk, w, M, nchunks, k);
    return count_from_first(stage_blk[0], stage_blk[1], stage_blk + 2, blk, w, M, c0, nchunks, k, planes);
}

// Settle and emit the candidates of one warp tile (cand[g] bit w: window
// 32*(tile*32G + 32g + lane) + w; the tile still staged at `stage`, from
// block tile*32G + d.c0 on) with the whole warp working on them together,
// whichever lanes they came from: the candidates are written, in window
// order, to the warp's queue q in shared memory (kQueueCap entries); each
// lane then counts every 32nd of them exactly (up to k), the hits are
// compacted in place, in window order, and written once to tmp behind one
// warp-aggregated atomic on cursor (coalesced); *entry receives {hits,
// first}.  A lane that held candidates in one group of a tile would
// otherwise keep the other 31 lanes waiting while it counts them one by one.
// Returns false, having done nothing, when the tile has more than kQueueCap
// candidates or k is too large for a count to share 32 bits with its
// window.  Call with the whole warp.
template <int G>
__device__ __forceinline__ bool settle_emit_queued(const uint32_t (&cand)[G], uint32_t tile,
                                                   const uint2 *stage, uint32_t *q, const PatDesc &d,
                                                   const uint4 *__restrict__ M,
                                                   const uint2 *__restrict__ planes,
                                                   const uint32_t *__restrict__ unk,
                                                   pm_hit *__restrict__ tmp, uint64_t cap,
                                                   unsigned long long *__restrict__ cursor,
                                                   TileEntry *entry)
{
    static_assert(G == 4 || G == 8, "one byte per group, four groups per word");
    constexpr int NW = G / 4;                        // words of packed group counts
    constexpr uint32_t kWinBits = G == 4 ? 12u : 13u;  // window within the tile
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t k = (uint32_t)d.k;
    // byte j of word i: this lane's candidates in group 4i + j (at most 32 each)
    uint32_t packed[NW];
    uint32_t mine = 0;
#pragma unroll
    for (int i = 0; i < NW; ++i) {
        packed[i] = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) packed[i] |= (uint32_t)__popc(cand[4 * i + j]) << (8 * j);
        mine += (packed[i] * 0x01010101u) >> 24;  // sum of the bytes (at most 128)
    }
    const uint32_t total = __reduce_add_sync(kFull, mine);
    if (total > kQueueCap || k >= (1u << (32u - kWinBits))) return false;
    // Inclusive scans over the lanes of four bytes at once: no byte ever
    // exceeds total <= 255, so bytes never carry into each other.
    uint32_t pos[NW];
    uint32_t before = 0;  // candidates of the groups of earlier words
#pragma unroll
    for (int i = 0; i < NW; ++i) {
        uint32_t incl = packed[i];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t v = __shfl_up_sync(kFull, incl, o);
            if (lane >= (uint32_t)o) incl += v;
        }
        const uint32_t tot = __shfl_sync(kFull, incl, 31);
        // byte j: where this lane's candidates of group 4i + j start (all of
        // the earlier groups, then those of this group on earlier lanes)
        pos[i] = before * 0x01010101u + tot * 0x01010100u + (incl - packed[i]);
        before += (tot * 0x01010101u) >> 24;
    }
#pragma unroll
    for (int g = 0; g < G; ++g) {
        uint32_t p = (pos[g / 4] >> (8 * (g % 4))) & 0xffu;
        uint32_t m = cand[g];
        while (m) {
            const uint32_t w = __ffs(m) - 1;
            m &= m - 1;
            q[p++] = ((uint32_t)g << 10) | (lane << 5) | w;  // window within the tile
        }
    }
    __syncwarp();
    uint32_t hits = 0;
    for (uint32_t i0 = 0; i0 < total; i0 += 32) {
        const uint32_t i = i0 + lane;
        uint32_t rec = 0;
        bool hit = false;
        if (i < total) {
            const uint32_t e = q[i];
            const uint32_t gl = e >> 5;  // block within the tile
            const uint32_t c = candidate_count(stage + gl, (uint64_t)tile * (32u * G) + gl, e & 31u, M, d.c0,
                                               d.nchunks, k, planes, unk);
            hit = c <= k;
            rec = e | (c << kWinBits);
        }
        const uint32_t hb = __ballot_sync(kFull, hit);
        __syncwarp();  // every entry of this round is read before any is overwritten
        if (hit) q[hits + __popc(hb & ((1u << lane) - 1u))] = rec;
        hits += __popc(hb);
    }
    unsigned long long base = 0;
    if (hits) {
        __syncwarp();
        if (lane == 0) base = atomicAdd(cursor, (unsigned long long)hits);
        base = __shfl_sync(kFull, base, 0);
        const uint64_t w0 = (uint64_t)tile * (1024u * G);
        for (uint32_t i = lane; i < hits; i += 32) {
            const uint32_t r = q[i];
            if (base + i < cap)
                tmp[base + i] = pm_hit{(uint32_t)(w0 + (r & ((1u << kWinBits) - 1u))), r >> kWinBits};
        }
    }
    if (lane == 0) *entry = TileEntry{hits, (uint32_t)base};
    __syncwarp();  // the queue is rewritten by the next tile
    return true;
}

}  // namespace scan
}  // namespace pm
